// kf_pchain.cu -- the paper's own chain (Table II / Table IV): K1 convert RGBA to gray,
// K2 IIR filter, K3 Gaussian smoothing, K4 gradient filter, K5 threshold computation,
// any contiguous group of them fused into one kernel (Sec. V-B, Eq. 2), and K6, the
// Kalman filter over feature positions, after the kernel-to-kernel dependency.
//
// A group (0-based stages A..B) works on 32 x 32 tiles of its input (lane = column); a
// group with K3 and K4 has a 2-pixel halo and writes the inner 28 x 28 (30 x 30 with one
// of them). Horizontal taps are warp shuffles. pc_kernel<A, B>, for groups without K2:
// one warp per (tile, frame) streams the 32 rows in registers. pc_temporal_kernel<A, B>,
// for groups holding K2 (the IIR filter, a recursion over frames): one block of 4 warps
// per tile walks every frame of the video in order, each warp keeping the filter state of
// its 8 rows in registers and loading the next frame's rows while it computes this one;
// the spatial stages exchange rows through shared memory. No filter state goes through
// memory.
//
// Clamp-to-edge per stage: the group's input is read at clamped coordinates, which is
// the clamp of K1..K3's inputs (point stages commute with it). K4 reads K3's output at
// clamped coordinates: in a tile at a frame edge the out-of-frame columns of G' take the
// edge column's value (shuffle), and at the frame's first and last rows the Sobel's
// vertical neighbour is the row itself.
//
// Units (exact where the values are integers): Y' = 77 R + 150 G + 29 B (scale 65280),
// y' (scale 65280, FP32 recursion), G' = [1 2 1] x [1 2 1] of y' (scale 16 * 65280),
// M' = |Sobel x| + |Sobel y| of G' (same scale), mask = M' > 0.25 * 16 * 65280. Every
// stage is one device function shared by all groups, so partitions agree bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "kf_ctx.h"

namespace kf {
int ctx_device(const kf_ctx *ctx);  // kf_api.cu
}

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int TS = 32;   // tile side: 32 lanes x 32 streamed rows of the group's input
constexpr int WPB = 4;   // warps per block of the per-frame groups
constexpr int NREG = KF_PC_REGIONS;
constexpr int GRIDN = 4;  // regions per side
constexpr float ALPHA = 0.25f;
constexpr float TAU = 0.25f * 16.0f * 65280.0f;  // threshold on M' (exact in FP32)
constexpr double KQ = 0.5, KR = 4.0, KP0 = 100.0;  // Kalman: process noise, measurement noise, initial velocity variance
constexpr int CHUNK = KF_PC_CHUNK;  // frames per chunk of the IIR recursion
// Per-frame sums (the mask count and the 16 regions' count, sum x, sum y) are added into
// one of NSLOT copies per frame, chosen by the warp, and the copies are summed afterwards:
// every warp of a frame adding to the same 49 counters serialised the atomics in L2.
constexpr int NSLOT = 32;
constexpr int NCNT = 1 + 3 * NREG;

struct PcParams {
    const uint32_t *in;   // RGBA pixels (A == 0) or FP32 bit patterns
    int64_t in_pitch, in_fstride;    // elements
    void *out;            // FP32 map (B < 4) or u8 mask (B == 4)
    int64_t out_pitch, out_fstride;  // elements
    int W, H, T;
    int tiles_x, tiles_y;
    int32_t *counts, *regions;       // B == 4: the final sums
    int32_t *slots;                  // B == 4: [T][NSLOT][NCNT] partial sums, zeroed before the launch
    float *state;                    // IIR states at the chunk starts: [n_chunks][H][state_pitch]
    int64_t state_pitch;
    int n_chunks;                    // ceil(T / CHUNK)
    float decay_chunk;               // (1 - ALPHA)^CHUNK in FP32
};

// ---- the stages (one definition each, used by every group)
__device__ __forceinline__ float k1_gray(uint32_t rgba)
{
    const float r = (float)(rgba & 0xffu), g = (float)((rgba >> 8) & 0xffu), b = (float)((rgba >> 16) & 0xffu);
    return fmaf(29.0f, b, fmaf(150.0f, g, 77.0f * r));  // integer <= 65280: exact
}
__device__ __forceinline__ float k2_iir(float prev, float Y) { return fmaf(ALPHA, Y - prev, prev); }
// [1 2 1] of three neighbours (the centre weighted 2)
__device__ __forceinline__ float tap121(float l, float c, float r) { return fmaf(2.0f, c, l + r); }

template <int A, int B> struct Group {
    static constexpr bool H1 = A <= 1 && 1 <= B, H2 = A <= 2 && 2 <= B, H3 = A <= 3 && 3 <= B, H4 = B == 4;
    static constexpr int HALO = (H2 ? 1 : 0) + (H3 ? 1 : 0);
    static constexpr int OUT = TS - 2 * HALO;  // output tile side
    static constexpr bool TEMPORAL = H1;
};

// Groups without K2: one warp per (tile, frame).
template <int A, int B>
__global__ void __launch_bounds__(32 * WPB) pc_kernel(const PcParams p)
{
    using G = Group<A, B>;
    static_assert(!G::TEMPORAL, "groups holding the IIR filter run pc_temporal_kernel");
    constexpr int HALO = G::HALO, OUT = G::OUT;
    __shared__ int acc[WPB][NREG][3];  // this frame's region sums of the warp (B == 4)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t n_tiles = (int64_t)p.tiles_x * p.tiles_y;
    if (gw >= n_tiles * p.T) return;  // warp-uniform; no block barriers below
    const int64_t tile = gw % n_tiles;
    const int f_begin = (int)(gw / n_tiles), f_end = f_begin + 1;
    const int W = p.W, H = p.H;
    const int tx = (int)(tile % p.tiles_x), ty = (int)(tile / p.tiles_x);
    const int x = tx * OUT - HALO + lane;  // this lane's input column
    const int xc = min(max(x, 0), W - 1);
    const int y0 = ty * OUT - HALO;         // the tile's first input row
    const bool out_col = lane >= HALO && lane < TS - HALO && x < W;
    const bool edge_tile = (tx * OUT - HALO < 0) || (tx * OUT - HALO + TS > W);
    const int src_lane = lane + (xc - x);   // the lane holding the clamped column
    const int rxl = (GRIDN * xc) / W;      // region column of this lane
    if constexpr (G::H4) {
        if (lane < NREG) acc[wib][lane][0] = acc[wib][lane][1] = acc[wib][lane][2] = 0;
        __syncwarp();
    }

    uint32_t buf[TS];  // input rows of the next frame to process
    auto load = [&](int f, uint32_t (&v)[TS]) {
        const uint32_t *base = p.in + (int64_t)f * p.in_fstride + xc;
#pragma unroll
        for (int r = 0; r < TS; ++r) v[r] = __ldg(base + (int64_t)min(max(y0 + r, 0), H - 1) * p.in_pitch);
    };
    load(f_begin, buf);

    for (int f = f_begin; f < f_end; ++f) {
        uint32_t cur[TS];
#pragma unroll
        for (int r = 0; r < TS; ++r) cur[r] = buf[r];
        if (f + 1 < f_end) load(f + 1, buf);  // in flight while this frame computes
        float *outf = static_cast<float *>(p.out) + (int64_t)f * p.out_fstride;
        uint8_t *outm = static_cast<uint8_t *>(p.out) + (int64_t)f * p.out_fstride;
        [[maybe_unused]] float hy[TS], Gv[TS], D[TS], S[TS];
        [[maybe_unused]] unsigned count = 0;

        // the output row o of the group's last stage (tile row, global row y0 + o)
        auto emit = [&](int o, float v) {
            const int gy = y0 + o;
            if (gy >= H) return;  // rows past the frame (warp-uniform)
            if constexpr (!G::H4) {
                if (out_col) outf[(int64_t)gy * p.out_pitch + x] = v;
            } else {
                const bool m = out_col && v > TAU;
                if (out_col) outm[(int64_t)gy * p.out_pitch + x] = (uint8_t)m;
                count += __popc(__ballot_sync(FULLM, m));
                if (m) {
                    const int rg = ((GRIDN * gy) / H) * GRIDN + rxl;
                    atomicAdd(&acc[wib][rg][0], 1);
                    atomicAdd(&acc[wib][rg][1], x);
                    atomicAdd(&acc[wib][rg][2], gy);
                }
            }
        };
        // K4 (+ K5) at tile row o from D, S of rows o-1, o, o+1; at the frame's first and
        // last rows the missing neighbour is the row itself (clamp on G')
        auto sobel_out = [&](int o, float Dm, float Dc, float Dp, float Sm, float Sc, float Sp) {
            const int gy = y0 + o;
            const float dm = gy - 1 < 0 ? Dc : Dm, dp = gy + 1 > H - 1 ? Dc : Dp;
            const float sm = gy - 1 < 0 ? Sc : Sm, sp = gy + 1 > H - 1 ? Sc : Sp;
            const float gx = tap121(dm, Dc, dp);
            const float gyv = sp - sm;
            emit(o, fabsf(gx) + fabsf(gyv));
        };
        // K3's output row q of the tile: the column clamp, then the Sobel's row partials
        auto push_G = [&](int q, float g) {
            if constexpr (G::H2)
                if (edge_tile) g = __shfl_sync(FULLM, g, src_lane);
            Gv[q] = g;
            const float gl = __shfl_up_sync(FULLM, g, 1), gr = __shfl_down_sync(FULLM, g, 1);
            D[q] = gr - gl;
            S[q] = tap121(gl, g, gr);
        };

#pragma unroll
        for (int r = 0; r < TS; ++r) {
            const uint32_t v = cur[r];
            if constexpr (A == 0) {
                emit(r, k1_gray(v));  // K1 alone (a group from K1 on that holds K2 is temporal)
            } else if constexpr (A == 2) {
                const float yv = __uint_as_float(v);
                // ---- K3: horizontal [1 2 1], then vertical [1 2 1] one row behind
                hy[r] = tap121(__shfl_up_sync(FULLM, yv, 1), yv, __shfl_down_sync(FULLM, yv, 1));
                if (r >= 2) {
                    const int q = r - 1;
                    const float g = tap121(hy[q - 1], hy[q], hy[q + 1]);
                    if constexpr (B == 2) {
                        emit(q, g);
                    } else {
                        push_G(q, g);
                        // output rows 2..29: G rows 1..30 exist
                        if (q >= 3) sobel_out(q - 1, D[q - 2], D[q - 1], D[q], S[q - 2], S[q - 1], S[q]);
                    }
                }
            } else if constexpr (A == 3) {
                push_G(r, __uint_as_float(v));
                if (r >= 2) sobel_out(r - 1, D[r - 2], D[r - 1], D[r], S[r - 2], S[r - 1], S[r]);
            } else {
                emit(r, __uint_as_float(v));  // K5 alone on M'
            }
        }

        if constexpr (G::H4) {
            __syncwarp();
            int32_t *sl = p.slots + ((int64_t)f * NSLOT + (int)(gw % NSLOT)) * NCNT;
            if (lane == 0 && count) atomicAdd(sl, (int)count);
            if (lane < NREG) {
                int *a = acc[wib][lane];
                if (a[0]) {
                    atomicAdd(sl + 1 + 3 * lane + 0, a[0]);
                    atomicAdd(sl + 1 + 3 * lane + 1, a[1]);
                    atomicAdd(sl + 1 + 3 * lane + 2, a[2]);
                    a[0] = a[1] = a[2] = 0;
                }
            }
            __syncwarp();
        }
    }
}

// Groups holding K2: one block of 4 warps per tile walks every frame of the video in
// order. Warp w owns tile rows 8w .. 8w+7 for the point stages (its 8 IIR states per lane
// stay in registers; the next frame's 8 input rows are loaded while this frame computes),
// then the spatial stages read neighbouring rows through shared memory (y', then G'), two
// block barriers per frame. Four warps per tile give the recursion 4x the warps of one
// warp per tile.
constexpr int TW = 4;        // warps per tile
constexpr int RW = TS / TW;  // rows per warp

template <int A, int B>
__global__ void __launch_bounds__(32 * TW) pc_temporal_kernel(const PcParams p)
{
    // blockIdx.y: the chunk of CHUNK frames; the filter starts from the state the carry
    // pass left for the frame before the chunk (at clamped coordinates, like the input)
    using G = Group<A, B>;
    static_assert(G::TEMPORAL, "groups holding the IIR filter");
    constexpr int HALO = G::HALO, OUT = G::OUT;
    __shared__ float ys[TS][TS];  // y' of the tile (B >= 2)
    __shared__ float gs[TS][TS];  // G' of the tile (B >= 3)
    __shared__ int acc[TW][NREG][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x;
    const int W = p.W, H = p.H;
    const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
    const int x = tx * OUT - HALO + lane;
    const int xc = min(max(x, 0), W - 1);
    const int y0 = ty * OUT - HALO;
    const bool out_col = lane >= HALO && lane < TS - HALO && x < W;
    const bool edge_tile = (tx * OUT - HALO < 0) || (tx * OUT - HALO + TS > W);
    const int src_lane = lane + (xc - x);
    const int rxl = (GRIDN * xc) / W;
    const int r0 = RW * w;  // this warp's first tile row
    const int f0 = blockIdx.y * CHUNK, f1 = min(f0 + CHUNK, p.T);
    if constexpr (G::H4) {
        if (lane < NREG) acc[w][lane][0] = acc[w][lane][1] = acc[w][lane][2] = 0;
        __syncwarp();
    }
    uint32_t buf[RW];
    auto load = [&](int f) {
        const uint32_t *base = p.in + (int64_t)f * p.in_fstride + xc;
#pragma unroll
        for (int i = 0; i < RW; ++i) buf[i] = __ldg(base + (int64_t)min(max(y0 + r0 + i, 0), H - 1) * p.in_pitch);
    };
    float st[RW];
    {
        const float *s0 = p.state + (int64_t)blockIdx.y * H * p.state_pitch + xc;
#pragma unroll
        for (int i = 0; i < RW; ++i) st[i] = s0[(int64_t)min(max(y0 + r0 + i, 0), H - 1) * p.state_pitch];
    }
    load(f0);
    for (int f = f0; f < f1; ++f) {
        uint32_t cur[RW];
#pragma unroll
        for (int i = 0; i < RW; ++i) cur[i] = buf[i];
        if (f + 1 < f1) load(f + 1);
        float *outf = static_cast<float *>(p.out) + (int64_t)f * p.out_fstride;
        uint8_t *outm = static_cast<uint8_t *>(p.out) + (int64_t)f * p.out_fstride;
        [[maybe_unused]] unsigned count = 0;
        auto emit = [&](int o, float v) {  // tile row o (warp-uniform)
            const int gy = y0 + o;
            if (gy >= H) return;
            if constexpr (!G::H4) {
                if (out_col) outf[(int64_t)gy * p.out_pitch + x] = v;
            } else {
                const bool m = out_col && v > TAU;
                if (out_col) outm[(int64_t)gy * p.out_pitch + x] = (uint8_t)m;
                count += __popc(__ballot_sync(FULLM, m));
                if (m) {
                    const int rg = ((GRIDN * gy) / H) * GRIDN + rxl;
                    atomicAdd(&acc[w][rg][0], 1);
                    atomicAdd(&acc[w][rg][1], x);
                    atomicAdd(&acc[w][rg][2], gy);
                }
            }
        };
        // ---- K1, K2 on this warp's rows
#pragma unroll
        for (int i = 0; i < RW; ++i) {
            const float Y = A == 0 ? k1_gray(cur[i]) : __uint_as_float(cur[i]);
            st[i] = k2_iir(st[i], Y);
            if constexpr (B == 1) emit(r0 + i, st[i]);
            else ys[r0 + i][lane] = st[i];
        }
        if constexpr (B >= 2) {
            __syncthreads();
            // ---- K3 on rows q of this warp with both neighbours in the tile (1..30)
            float hy[RW + 2];
#pragma unroll
            for (int i = 0; i < RW + 2; ++i) {
                const int r = r0 - 1 + i;
                if (r >= 0 && r < TS) {  // warp-uniform
                    const float yv = ys[r][lane];
                    hy[i] = tap121(__shfl_up_sync(FULLM, yv, 1), yv, __shfl_down_sync(FULLM, yv, 1));
                }
            }
#pragma unroll
            for (int i = 0; i < RW; ++i) {
                const int q = r0 + i;
                if (q < 1 || q > TS - 2) continue;
                float g = tap121(hy[i], hy[i + 1], hy[i + 2]);
                if constexpr (B == 2) {
                    emit(q, g);
                } else {
                    if (edge_tile) g = __shfl_sync(FULLM, g, src_lane);
                    gs[q][lane] = g;
                }
            }
            if constexpr (B >= 3) {
                __syncthreads();
                // ---- K4 (+ K5) on output rows o of this warp (2..29)
                float Dv[RW + 2], Sv[RW + 2];
#pragma unroll
                for (int i = 0; i < RW + 2; ++i) {
                    const int r = r0 - 1 + i;
                    if (r >= 1 && r <= TS - 2) {
                        const float g = gs[r][lane];
                        const float gl = __shfl_up_sync(FULLM, g, 1), gr = __shfl_down_sync(FULLM, g, 1);
                        Dv[i] = gr - gl;
                        Sv[i] = tap121(gl, g, gr);
                    }
                }
#pragma unroll
                for (int i = 0; i < RW; ++i) {
                    const int o = r0 + i;
                    if (o < 2 || o > TS - 3) continue;
                    const int gy = y0 + o;
                    const float dm = gy - 1 < 0 ? Dv[i + 1] : Dv[i], dp = gy + 1 > H - 1 ? Dv[i + 1] : Dv[i + 2];
                    const float sm = gy - 1 < 0 ? Sv[i + 1] : Sv[i], sp = gy + 1 > H - 1 ? Sv[i + 1] : Sv[i + 2];
                    emit(o, fabsf(tap121(dm, Dv[i + 1], dp)) + fabsf(sp - sm));
                }
            }
        }
        if constexpr (G::H4) {
            __syncwarp();
            int32_t *sl = p.slots + ((int64_t)f * NSLOT + (int)((blockIdx.x * TW + w) % NSLOT)) * NCNT;
            if (lane == 0 && count) atomicAdd(sl, (int)count);
            if (lane < NREG) {
                int *a = acc[w][lane];
                if (a[0]) {
                    atomicAdd(sl + 1 + 3 * lane + 0, a[0]);
                    atomicAdd(sl + 1 + 3 * lane + 1, a[1]);
                    atomicAdd(sl + 1 + 3 * lane + 2, a[2]);
                    a[0] = a[1] = a[2] = 0;
                }
            }
            __syncwarp();
        }
    }
}

// ---- the IIR recursion cut into chunks of CHUNK frames, so that chunks run in parallel.
// The filter is linear: started from state s before frame t0, y_{t0+j} = (1 - ALPHA)^(j+1) s
// + l_{t0+j}, where l is the same recursion started from 0. (1) Per chunk and pixel, l at
// the chunk's last frame; (2) per pixel, in chunk order, the state before each chunk:
// s_0 = Y_0 (so that y_0 = Y_0), s_k = (1 - ALPHA)^CHUNK s_{k-1} + l_end(k-1); (3) every
// group holding K2 runs each chunk from its s_k. The states are one FP32 plane per chunk;
// pass (2) overwrites l_end(k-1) with s_{k-1} in place.
template <int A0>  // 0: RGBA frames, 1: Y' map
__global__ void __launch_bounds__(32 * TW) pc_iir_local_kernel(const PcParams p)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = blockIdx.x * TS + lane;
    const int y = blockIdx.z * TS + RW * w;
    const int k = blockIdx.y;  // chunk (all but the last)
    if (x >= p.W) return;      // no block barriers here
    const int f0 = k * CHUNK;
    float l[RW];
#pragma unroll
    for (int i = 0; i < RW; ++i) l[i] = 0.0f;
    const uint32_t *base = p.in + x;
    const int nrows = min(RW, p.H - y);
#pragma unroll 4
    for (int f = f0; f < f0 + CHUNK; ++f) {  // unrolled: later frames' loads issue early
        const uint32_t *fr = base + (int64_t)f * p.in_fstride;
        uint32_t v[RW];
#pragma unroll
        for (int i = 0; i < RW; ++i) v[i] = i < nrows ? __ldg(fr + (int64_t)(y + i) * p.in_pitch) : 0u;
#pragma unroll
        for (int i = 0; i < RW; ++i) l[i] = k2_iir(l[i], A0 == 0 ? k1_gray(v[i]) : __uint_as_float(v[i]));
    }
    float *o = p.state + (int64_t)k * p.H * p.state_pitch + x;
#pragma unroll
    for (int i = 0; i < RW; ++i)
        if (y + i < p.H) o[(int64_t)(y + i) * p.state_pitch] = l[i];
}

template <int A0>
__global__ void pc_iir_carry_kernel(const PcParams p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)p.W * p.H) return;
    const int y = (int)(i / p.W), x = (int)(i - (int64_t)y * p.W);
    const uint32_t v = p.in[(int64_t)y * p.in_pitch + x];  // frame 0
    float s = A0 == 0 ? k1_gray(v) : __uint_as_float(v);
    float *col = p.state + (int64_t)y * p.state_pitch + x;
    const int64_t plane = (int64_t)p.H * p.state_pitch;
    // eight chunks' end states are loaded at once (independent loads), then carried
    for (int k0 = 1; k0 < p.n_chunks; k0 += 8) {
        float e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) e[j] = k0 + j < p.n_chunks ? col[(int64_t)(k0 + j - 1) * plane] : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            if (k0 + j < p.n_chunks) {
                col[(int64_t)(k0 + j - 1) * plane] = s;
                s = fmaf(p.decay_chunk, s, e[j]);
            }
        }
    }
    col[(int64_t)(p.n_chunks - 1) * plane] = s;
}

// the per-frame sums: counts[f] and regions[f][r][c] from the NSLOT partial copies
__global__ void pc_sums_kernel(const int32_t *slots, int T, int32_t *counts, int32_t *regions)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)T * NCNT) return;
    const int f = (int)(i / NCNT), j = (int)(i - (int64_t)f * NCNT);
    const int32_t *s = slots + (int64_t)f * NSLOT * NCNT + j;
    int tot = 0;
#pragma unroll 8
    for (int k = 0; k < NSLOT; ++k) tot += s[k * NCNT];
    if (j == 0) counts[f] = tot;
    else regions[(int64_t)f * 3 * NREG + (j - 1)] = tot;
}

// K6: one thread per track walks the frames. The constant-velocity model is the same per
// axis and starts from the same covariance, so the x and y axes share one symmetric 2 x 2
// covariance (P00 position, P01, P11 velocity) -- the block structure of the 4 x 4 filter.
__global__ void pc_kalman_kernel(const int32_t *regions, int T, int n, double *states, int32_t *status)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    bool started = false;
    double px = 0, py = 0, vx = 0, vy = 0, P00 = 0, P01 = 0, P11 = 0;
    for (int t = 0; t < T; ++t) {
        const int32_t *rg = regions + ((int64_t)t * n + k) * 3;
        const int cnt = rg[0];
        const double zx = cnt > 0 ? (double)rg[1] / cnt : 0.0, zy = cnt > 0 ? (double)rg[2] / cnt : 0.0;
        int s;
        if (!started) {
            if (cnt > 0) {
                started = true;
                px = zx;
                py = zy;
                vx = vy = 0.0;
                P00 = KR;
                P01 = 0.0;
                P11 = KP0;
                s = 1;
            } else {
                s = 0;
            }
        } else {
            // predict: state by F, P by F P F' + Q with Q = q [[1/3, 1/2], [1/2, 1]]
            px += vx;
            py += vy;
            const double a = P00 + 2.0 * P01 + P11 + KQ / 3.0, b = P01 + P11 + KQ / 2.0, c = P11 + KQ;
            P00 = a;
            P01 = b;
            P11 = c;
            if (cnt > 0) {
                const double Sd = P00 + KR, k0 = P00 / Sd, k1 = P01 / Sd;
                const double ex = zx - px, ey = zy - py;
                px += k0 * ex;
                vx += k1 * ex;
                py += k0 * ey;
                vy += k1 * ey;
                P11 -= k1 * P01;
                P01 *= 1.0 - k0;
                P00 *= 1.0 - k0;
                s = 1;
            } else {
                s = 2;
            }
        }
        double *o = states + ((int64_t)t * n + k) * 4;
        o[0] = px;
        o[1] = py;
        o[2] = vx;
        o[3] = vy;
        status[(int64_t)t * n + k] = s;
    }
}

template <int A, int B>
int launch_one(const PcParams &p, cudaStream_t s)
{
    using G = Group<A, B>;
    const int64_t n_tiles = (int64_t)p.tiles_x * p.tiles_y;
    if constexpr (G::TEMPORAL) {
        // the chunk states first: local ends, then the carry (in place)
        const dim3 lg((unsigned)((p.W + TS - 1) / TS), (unsigned)(p.n_chunks - 1), (unsigned)((p.H + TS - 1) / TS));
        if (p.n_chunks > 1) pc_iir_local_kernel<A><<<lg, 32 * TW, 0, s>>>(p);
        const int64_t px = (int64_t)p.W * p.H;
        pc_iir_carry_kernel<A><<<(unsigned)((px + 255) / 256), 256, 0, s>>>(p);
        pc_temporal_kernel<A, B><<<dim3((unsigned)n_tiles, (unsigned)p.n_chunks), 32 * TW, 0, s>>>(p);
    } else {
        const int64_t warps = n_tiles * p.T;
        pc_kernel<A, B><<<(unsigned)((warps + WPB - 1) / WPB), 32 * WPB, 0, s>>>(p);
    }
    return (int)cudaGetLastError();
}

int launch_group(int a, int b, const PcParams &p, cudaStream_t s)
{
#define KF_PC_CASE(A, B) \
    if (a == A && b == B) return launch_one<A, B>(p, s);
    KF_PC_CASE(0, 0) KF_PC_CASE(0, 1) KF_PC_CASE(0, 2) KF_PC_CASE(0, 3) KF_PC_CASE(0, 4)
    KF_PC_CASE(1, 1) KF_PC_CASE(1, 2) KF_PC_CASE(1, 3) KF_PC_CASE(1, 4)
    KF_PC_CASE(2, 2) KF_PC_CASE(2, 3) KF_PC_CASE(2, 4)
    KF_PC_CASE(3, 3) KF_PC_CASE(3, 4)
    KF_PC_CASE(4, 4)
#undef KF_PC_CASE
    return (int)cudaErrorInvalidValue;
}

int halo_of(int a, int b) { return (a <= 2 && 2 <= b ? 1 : 0) + (a <= 3 && 3 <= b ? 1 : 0); }

kf_status fail(kf_ctx *c, int e)
{
    c->last_cuda = e;
    return KF_ECUDA;
}

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

int64_t ws_pitch(int64_t W) { return (W + 7) / 8 * 8; }

// bytes per pixel of the map stage k writes (k = -1: the RGBA frames)
double map_bytes(int k) { return k < 0 ? 4.0 : (k == 4 ? 1.0 : 4.0); }

// the int32 region sums of x (and y) stay exact: at most max(W, H) * (W H / 16 + W + H)
bool sums_fit(int64_t W, int64_t H) { return (W > H ? W : H) * (W * H / 16 + W + H) < 0x7fffffffLL; }

kf_status check_video(const kf_pc_video *v)
{
    if (!v || !v->rgba || v->W <= 0 || v->H <= 0 || v->T < 0 || v->pitch < v->W || !aligned(v->rgba, 16)) return KF_EINVAL;
    if (v->W > (1 << 24) || v->H > (1 << 24) || v->T > 0x7fffffff || v->W * v->H > 0x7fffffffLL) return KF_EINVAL;
    if (!sums_fit(v->W, v->H)) return KF_EINVAL;
    return KF_OK;
}
kf_status check_out(const kf_pc_out *o, int64_t W)
{
    if (!o || !o->mask || o->mask_pitch < W || !o->counts || !o->regions || !aligned(o->counts, 4) ||
        !aligned(o->regions, 4))
        return KF_EINVAL;
    return KF_OK;
}

PcParams params_for(int a, int b, int64_t W, int64_t H, int64_t T)
{
    PcParams p{};
    const int out = TS - 2 * halo_of(a, b);
    p.W = (int)W;
    p.H = (int)H;
    p.T = (int)T;
    p.tiles_x = (int)((W + out - 1) / out);
    p.tiles_y = (int)((H + out - 1) / out);
    return p;
}

int64_t n_chunks(int64_t T) { return (T + KF_PC_CHUNK - 1) / KF_PC_CHUNK; }
// bytes of the IIR chunk states: one FP32 plane per chunk (pitch round_up(W, 8)), 256-aligned
size_t state_bytes(int64_t W, int64_t H, int64_t T)
{
    return ((size_t)(n_chunks(T) * H * ws_pitch(W)) * sizeof(float) + 255) / 256 * 256;
}
bool holds_iir(int a, int b) { return a <= 1 && 1 <= b; }

// one group over prepared pointers; zeroes counts and regions first when it ends at K5;
// `state`: the chunk-state planes (groups holding K2)
size_t slot_bytes(int64_t T) { return ((size_t)T * NSLOT * NCNT * sizeof(int32_t) + 255) / 256 * 256; }

kf_status run_group(kf_ctx *ctx, int a, int b, const uint32_t *in, int64_t in_pitch, void *out, int64_t out_pitch,
                    int64_t W, int64_t H, int64_t T, int32_t *counts, int32_t *regions, float *state, int32_t *slots,
                    cudaStream_t s)
{
    if (T == 0) return KF_OK;
    PcParams p = params_for(a, b, W, H, T);
    p.state = state;
    p.state_pitch = ws_pitch(W);
    p.n_chunks = (int)n_chunks(T);
    p.decay_chunk = (float)pow(1.0 - 0.25, (double)KF_PC_CHUNK);
    p.in = in;
    p.in_pitch = in_pitch;
    p.in_fstride = in_pitch * H;
    p.out = out;
    p.out_pitch = out_pitch;
    p.out_fstride = out_pitch * H;
    p.counts = counts;
    p.regions = regions;
    p.slots = slots;
    if (b == 4) {
        const cudaError_t e = cudaMemsetAsync(slots, 0, sizeof(int32_t) * NSLOT * NCNT * (size_t)T, s);
        if (e != cudaSuccess) return fail(ctx, (int)e);
    }
    const int64_t n_tiles = (int64_t)p.tiles_x * p.tiles_y;
    const bool temporal = holds_iir(a, b);
    if ((temporal ? n_tiles : (n_tiles * T + WPB - 1) / WPB) > 0x7fffffffLL) return KF_EINVAL;
    if (temporal && (p.n_chunks > 65535 || (H + TS - 1) / TS > 65535)) return KF_EINVAL;
    int e = launch_group(a, b, p, s);
    if (!e && b == 4) {
        const int64_t n = T * NCNT;
        pc_sums_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(slots, (int)T, counts, regions);
        e = (int)cudaGetLastError();
    }
    return e ? fail(ctx, e) : KF_OK;
}

}  // namespace

extern "C" {

kf_status kf_pc_traffic(kf_ctx *ctx, uint32_t cuts, int64_t W, int64_t H, int64_t T, double *bytes)
{
    if (!ctx || !bytes || W <= 0 || H <= 0 || T < 0 || cuts >= 16) return KF_EINVAL;
    const double px = (double)W * H * T;
    double tot = 0;
    int a = 0;
    for (int i = 0; i < KF_PC_STAGES; ++i) {
        if (i == KF_PC_STAGES - 1 || (cuts >> i & 1)) {
            const int out = TS - 2 * halo_of(a, i);
            const double read_factor = (double)TS * TS / ((double)out * out);
            tot += px * (map_bytes(a - 1) * read_factor + map_bytes(i));
            if (holds_iir(a, i)) {
                // the chunked recursion: the local pass reads all but the last chunk and writes
                // their end states; the carry reads frame 0 and those states and writes every
                // chunk's start state; the group reads the start states with its halo
                const double hw = (double)W * H, nc = (double)n_chunks(T);
                tot += (nc - 1) * KF_PC_CHUNK * hw * map_bytes(a - 1) + (nc - 1) * hw * 4.0;
                tot += hw * map_bytes(a - 1) + (nc - 1) * hw * 4.0 + nc * hw * 4.0;
                tot += nc * hw * 4.0 * read_factor;
            }
            a = i + 1;
        }
    }
    tot += (double)T * 4.0 * (1 + 3 * NREG);  // counts and region sums
    *bytes = tot;
    return KF_OK;
}

kf_status kf_pc_plan(kf_ctx *ctx, int64_t W, int64_t H, int64_t T, uint32_t *cuts, double *bytes)
{
    if (!ctx || !cuts) return KF_EINVAL;
    double best = 0;
    uint32_t arg = 0;
    for (uint32_t c = 0; c < 16; ++c) {
        double b = 0;
        const kf_status s = kf_pc_traffic(ctx, c, W, H, T, &b);
        if (s != KF_OK) return s;
        if (c == 0 || b < best) {
            best = b;
            arg = c;
        }
    }
    *cuts = arg;
    if (bytes) *bytes = best;
    return KF_OK;
}

kf_status kf_pc_workspace_bytes(kf_ctx *ctx, uint32_t cuts, int64_t W, int64_t H, int64_t T, size_t *bytes)
{
    if (!ctx || !bytes || W <= 0 || H <= 0 || T < 0 || cuts >= 16) return KF_EINVAL;
    const int n_cuts = __builtin_popcount(cuts);
    const size_t plane = (size_t)(ws_pitch(W) * H * T) * sizeof(float);
    const size_t plane_a = (plane + 255) / 256 * 256;
    *bytes = state_bytes(W, H, T) + slot_bytes(T) + (n_cuts == 0 ? 0 : (n_cuts == 1 ? plane_a : 2 * plane_a));
    return KF_OK;
}

kf_status kf_pc_run(kf_ctx *ctx, uint32_t cuts, const kf_pc_video *video, const kf_pc_out *out, void *workspace,
                    size_t workspace_bytes, void *stream)
{
    if (!ctx || cuts >= 16) return KF_EINVAL;
    kf_status st = check_video(video);
    if (st != KF_OK) return st;
    if ((st = check_out(out, video->W)) != KF_OK) return st;
    const int dev = kf::ctx_device(ctx);
    if (dev < 0) return KF_ESTATE;
    size_t need = 0;
    kf_pc_workspace_bytes(ctx, cuts, video->W, video->H, video->T, &need);
    if (need && (!workspace || !aligned(workspace, 256))) return KF_EINVAL;
    if (workspace_bytes < need) return KF_ENOMEM;
    if (cudaSetDevice(dev) != cudaSuccess) return KF_ECUDA;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t W = video->W, H = video->H, T = video->T, wp = ws_pitch(W);
    const size_t plane_a = ((size_t)(wp * H * T) * sizeof(float) + 255) / 256 * 256;
    float *state = static_cast<float *>(workspace);
    int32_t *slots = reinterpret_cast<int32_t *>(static_cast<char *>(workspace) + state_bytes(W, H, T));
    char *maps = reinterpret_cast<char *>(slots) + slot_bytes(T);
    float *planes[2] = {reinterpret_cast<float *>(maps), reinterpret_cast<float *>(maps + plane_a)};
    const uint32_t *in = reinterpret_cast<const uint32_t *>(video->rgba);
    int64_t in_pitch = video->pitch;
    int a = 0, k = 0;
    for (int i = 0; i < KF_PC_STAGES; ++i) {
        if (i != KF_PC_STAGES - 1 && !(cuts >> i & 1)) continue;
        const bool last = i == KF_PC_STAGES - 1;
        void *o = last ? static_cast<void *>(out->mask) : static_cast<void *>(planes[k % 2]);
        const int64_t op = last ? out->mask_pitch : wp;
        st = run_group(ctx, a, i, in, in_pitch, o, op, W, H, T, out->counts, out->regions, state, slots, s);
        if (st != KF_OK) return st;
        in = reinterpret_cast<const uint32_t *>(planes[k % 2]);
        in_pitch = wp;
        ++k;
        a = i + 1;
    }
    return KF_OK;
}

kf_status kf_pc_group_workspace_bytes(kf_ctx *ctx, int a, int b, int64_t W, int64_t H, int64_t T, size_t *bytes)
{
    if (!ctx || !bytes || a < 0 || b < a || b >= KF_PC_STAGES || W <= 0 || H <= 0 || T < 0) return KF_EINVAL;
    *bytes = (holds_iir(a, b) ? state_bytes(W, H, T) : 0) + (b == 4 ? slot_bytes(T) : 0);
    return KF_OK;
}

kf_status kf_pc_run_group(kf_ctx *ctx, int a, int b, const kf_pc_video *video, const float *in, int64_t in_pitch,
                          float *out, int64_t out_pitch, const kf_pc_out *out_mask, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    if (!ctx || a < 0 || b < a || b >= KF_PC_STAGES) return KF_EINVAL;
    // geometry from the video descriptor (its rgba is only read when a == 0)
    if (!video || video->W <= 0 || video->H <= 0 || video->T < 0 || video->T > 0x7fffffff || !sums_fit(video->W, video->H))
        return KF_EINVAL;
    const int64_t W = video->W, H = video->H, T = video->T;
    if (a == 0) {
        const kf_status st = check_video(video);
        if (st != KF_OK) return st;
    } else if (!in || in_pitch < W || !aligned(in, 4)) {
        return KF_EINVAL;
    }
    if (b == 4) {
        const kf_status st = check_out(out_mask, W);
        if (st != KF_OK) return st;
    } else if (!out || out_pitch < W || !aligned(out, 4)) {
        return KF_EINVAL;
    }
    const size_t need = (holds_iir(a, b) ? state_bytes(W, H, T) : 0) + (b == 4 ? slot_bytes(T) : 0);
    if (need) {
        if (!workspace || !aligned(workspace, 256)) return KF_EINVAL;
        if (workspace_bytes < need) return KF_ENOMEM;
    }
    const int dev = kf::ctx_device(ctx);
    if (dev < 0) return KF_ESTATE;
    if (cudaSetDevice(dev) != cudaSuccess) return KF_ECUDA;
    const uint32_t *src = a == 0 ? reinterpret_cast<const uint32_t *>(video->rgba) : reinterpret_cast<const uint32_t *>(in);
    const int64_t sp = a == 0 ? video->pitch : in_pitch;
    void *dst = b == 4 ? static_cast<void *>(out_mask->mask) : static_cast<void *>(out);
    const int64_t dp = b == 4 ? out_mask->mask_pitch : out_pitch;
    float *state = holds_iir(a, b) ? static_cast<float *>(workspace) : nullptr;
    int32_t *slots = b == 4 ? reinterpret_cast<int32_t *>(static_cast<char *>(workspace) +
                                                          (holds_iir(a, b) ? state_bytes(W, H, T) : 0))
                            : nullptr;
    return run_group(ctx, a, b, src, sp, dst, dp, W, H, T, b == 4 ? out_mask->counts : nullptr,
                     b == 4 ? out_mask->regions : nullptr, state, slots, static_cast<cudaStream_t>(stream));
}

kf_status kf_pc_kalman(kf_ctx *ctx, const int32_t *regions, int64_t T, int n_tracks, double *states, int32_t *status,
                       void *stream)
{
    if (!ctx || T < 0 || T > 0x7fffffff || n_tracks < 0) return KF_EINVAL;
    if (T == 0 || n_tracks == 0) return KF_OK;
    if (!regions || !states || !status || !aligned(regions, 4) || !aligned(states, 8) || !aligned(status, 4))
        return KF_EINVAL;
    const int dev = kf::ctx_device(ctx);
    if (dev < 0) return KF_ESTATE;
    if (cudaSetDevice(dev) != cudaSuccess) return KF_ECUDA;
    pc_kalman_kernel<<<(n_tracks + 63) / 64, 64, 0, static_cast<cudaStream_t>(stream)>>>(regions, (int)T, n_tracks,
                                                                                           states, status);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : fail(ctx, (int)e);
}

}  // extern "C"
