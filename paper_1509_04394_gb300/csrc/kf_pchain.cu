// kf_pchain.cu -- the paper's own chain (Table II / Table IV): K1 convert RGBA to gray,
// K2 IIR filter, K3 Gaussian smoothing, K4 gradient filter, K5 threshold computation,
// any contiguous group of them fused into one kernel (Sec. V-B, Eq. 2), and K6, the
// Kalman filter over feature positions, after the kernel-to-kernel dependency.
//
// A group (0-based stages A..B) runs pc_tile_kernel<A, B>: one block of 8 warps per tile
// of its input, 128 columns (4 per lane, 16-byte loads and stores) x 32 rows, each warp
// owning 4 rows for the point stages; K3 and K4 read neighbouring rows through shared
// memory and neighbouring columns by one shuffle per side. A group with K3 and K4 has a
// 2-row halo (its column halo is rounded up to one lane, 4 columns) and writes 120 x 28.
// Groups holding K2 (the IIR filter, a recursion over frames) run each tile over a chunk
// of frames from the chunk's start state (see the chunked recursion below), keeping each
// pixel's filter state in registers and loading the next frame's rows while computing
// this one; other groups run one (tile, frame) per block.
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
#include "kf_device.h"

namespace kf {
int ctx_device(const kf_ctx *ctx);  // kf_api.cu
}

namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int TS = 32;   // tile rows of the group's input
constexpr int C4 = 4;    // columns per lane
constexpr int TX = 32 * C4;  // tile columns
constexpr int TW = 8;        // warps per tile
constexpr int RW = TS / TW;  // rows per warp
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
    // 77 R + 150 G + 29 B in integers (<= 65280), placed under the exponent of 2^23 and
    // 2^23 subtracted: exact, and no conversion unit (a 4-byte dot product, __dp4a,
    // measured 15-20 % slower for the whole chain on this part)
    const uint32_t y = 77u * (rgba & 0xffu) + 150u * ((rgba >> 8) & 0xffu) + 29u * ((rgba >> 16) & 0xffu);
    return __uint_as_float(0x4B000000u | y) - 8388608.0f;
}
__device__ __forceinline__ float k2_iir(float prev, float Y) { return fmaf(ALPHA, Y - prev, prev); }
// [1 2 1] of three neighbours (the centre weighted 2)
__device__ __forceinline__ float tap121(float l, float c, float r) { return fmaf(2.0f, c, l + r); }

template <int A, int B> struct Group {
    static constexpr bool H1 = A <= 1 && 1 <= B, H2 = A <= 2 && 2 <= B, H3 = A <= 3 && 3 <= B, H4 = B == 4;
    static constexpr int HALO = (H2 ? 1 : 0) + (H3 ? 1 : 0);  // rows (and needed columns) each side
    static constexpr int HC = HALO ? 4 : 0;   // column halo, rounded to whole lanes (16-byte rows)
    static constexpr int OUTW = TX - 2 * HC;  // output tile: OUTW x OUTH
    static constexpr int OUTH = TS - 2 * HALO;
    static constexpr bool TEMPORAL = H1;
    // resident blocks per SM the register budget targets (measured: the fused filter with
    // spatial stages keeps its states and the next frame's rows in registers; at 3 blocks
    // of 8 warps it spilled 88-152 bytes and ran 9 % slower than at 2 without spills)
    static constexpr int MIN_BLOCKS = (H1 && HALO) ? 2 : 4;
};

// One block of TW = 8 warps per tile of TX = 128 columns (4 per lane) x TS = 32 rows of
// the group's input, over one frame, or over one chunk of CHUNK frames for a group holding
// K2. Warp w owns tile rows 4w .. 4w+3 for the point stages (and their IIR states, 16 per
// lane); K3 and K4 read the neighbouring rows through shared memory (y' then G'), with two
// block barriers per frame; horizontal taps are one shuffle per side per row.
template <int A, int B>
__global__ void __launch_bounds__(32 * TW, Group<A, B>::MIN_BLOCKS) pc_tile_kernel(const PcParams p)
{
    using G = Group<A, B>;
    constexpr int HALO = G::HALO, HC = G::HC, OUTW = G::OUTW, OUTH = G::OUTH;
    __shared__ float4 ys[TS][32];  // y' rows of the tile (groups with K3)
    __shared__ float4 gs[TS][32];  // G' rows of the tile (groups with K3 and K4)
    __shared__ int acc[TW][NREG][3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int tile = blockIdx.x;
    const int W = p.W, H = p.H;
    const int tx = tile % p.tiles_x, ty = tile / p.tiles_x;
    const int xt = tx * OUTW - HC;  // the tile's first input column (a multiple of 4)
    const int x0 = xt + C4 * lane;  // this lane's first column
    const int y0 = ty * OUTH - HALO;
    const int r0 = RW * w;
    // the lane's columns: clamped sources, and which are outputs
    const bool lane_inside = x0 >= 0 && x0 + C4 <= W;
    int xc[C4];
    unsigned out_bits = 0;
#pragma unroll
    for (int e = 0; e < C4; ++e) {
        xc[e] = min(max(x0 + e, 0), W - 1);
        const int col = C4 * lane + e;
        out_bits |= (col >= HC && col < TX - HC && x0 + e < W) ? (1u << e) : 0u;
    }
    const bool edge_tile = xt < 0 || xt + TX > W;
    const bool rows_inside = y0 >= 0 && y0 + TS <= H;
    [[maybe_unused]] const int rxl[C4] = {(GRIDN * xc[0]) / W, (GRIDN * xc[1]) / W, (GRIDN * xc[2]) / W,
                                          (GRIDN * xc[3]) / W};
    int f0, f1;
    if constexpr (G::TEMPORAL) {
        f0 = blockIdx.y * CHUNK;
        f1 = min(f0 + CHUNK, p.T);
    } else {
        f0 = blockIdx.y;
        f1 = f0 + 1;
    }
    if constexpr (G::H4) {
        if (lane < NREG) acc[w][lane][0] = acc[w][lane][1] = acc[w][lane][2] = 0;
        __syncwarp();
    }
    // 16-byte loads of one input row (4 columns), clamped columns at a frame edge
    auto load_row = [&](const uint32_t *plane, int64_t pitch, int r) {
        const uint32_t *row = plane + (int64_t)min(max(y0 + r, 0), H - 1) * pitch;
        uint4 v;
        if (lane_inside) {
            v = __ldg(reinterpret_cast<const uint4 *>(row + x0));
        } else {
            v.x = __ldg(row + xc[0]);
            v.y = __ldg(row + xc[1]);
            v.z = __ldg(row + xc[2]);
            v.w = __ldg(row + xc[3]);
        }
        return v;
    };
    uint4 buf[RW];
    auto load = [&](int f) {
        const uint32_t *plane = p.in + (int64_t)f * p.in_fstride;
#pragma unroll
        for (int i = 0; i < RW; ++i) buf[i] = load_row(plane, p.in_pitch, r0 + i);
    };
    [[maybe_unused]] float st[RW][C4];  // IIR states of this warp's rows (TEMPORAL)
    if constexpr (G::TEMPORAL) {
        const uint32_t *s0 = reinterpret_cast<const uint32_t *>(p.state) + (int64_t)blockIdx.y * H * p.state_pitch;
#pragma unroll
        for (int i = 0; i < RW; ++i) {
            const uint4 v = load_row(s0, p.state_pitch, r0 + i);
            st[i][0] = __uint_as_float(v.x);
            st[i][1] = __uint_as_float(v.y);
            st[i][2] = __uint_as_float(v.z);
            st[i][3] = __uint_as_float(v.w);
        }
    }
    load(f0);
    for (int f = f0; f < f1; ++f) {
        float *outf = static_cast<float *>(p.out) + (int64_t)f * p.out_fstride;
        uint8_t *outm = static_cast<uint8_t *>(p.out) + (int64_t)f * p.out_fstride;
        [[maybe_unused]] unsigned count = 0;
        // one output row of the group's last stage: 4 values of tile row o
        auto emit = [&](int o, const float (&v)[C4]) {
            const int gy = y0 + o;
            if (!rows_inside && gy >= H) return;  // warp-uniform
            if constexpr (!G::H4) {
                float *row = outf + (int64_t)gy * p.out_pitch + x0;
                if (out_bits == 0xfu) {
                    *reinterpret_cast<float4 *>(row) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int e = 0; e < C4; ++e) if (out_bits >> e & 1) row[e] = v[e];
                }
            } else {
                unsigned bits = 0;
#pragma unroll
                for (int e = 0; e < C4; ++e) bits |= (v[e] > TAU) ? (1u << e) : 0u;
                bits &= out_bits;
                uint8_t *row = outm + (int64_t)gy * p.out_pitch + x0;
                if (out_bits == 0xfu) {
                    *reinterpret_cast<uint32_t *>(row) = (bits & 1u) | (bits & 2u) << 7 | (bits & 4u) << 14 | (bits & 8u) << 21;
                } else {
#pragma unroll
                    for (int e = 0; e < C4; ++e) if (out_bits >> e & 1) row[e] = (uint8_t)(bits >> e & 1);
                }
                count += __popc(bits);
                if (bits) {
                    const int ry = ((GRIDN * gy) / H) * GRIDN;
#pragma unroll
                    for (int e = 0; e < C4; ++e) {
                        if (bits >> e & 1) {
                            const int rg = ry + rxl[e];
                            atomicAdd(&acc[w][rg][0], 1);
                            atomicAdd(&acc[w][rg][1], x0 + e);
                            atomicAdd(&acc[w][rg][2], gy);
                        }
                    }
                }
            }
        };
        // horizontal [1 2 1] of a row held 4 columns per lane (one shuffle per side)
        auto h121 = [&](const float4 v, float (&o)[C4]) {
            const float l = __shfl_up_sync(FULLM, v.w, 1), r = __shfl_down_sync(FULLM, v.x, 1);
            o[0] = tap121(l, v.x, v.y);
            o[1] = tap121(v.x, v.y, v.z);
            o[2] = tap121(v.y, v.z, v.w);
            o[3] = tap121(v.z, v.w, r);
        };

        // ---- the point stages on this warp's rows: K1, K2 (or the group's loaded input)
        [[maybe_unused]] float pv[RW][C4];
#pragma unroll
        for (int i = 0; i < RW; ++i) {
            const uint32_t u[C4] = {buf[i].x, buf[i].y, buf[i].z, buf[i].w};
#pragma unroll
            for (int e = 0; e < C4; ++e) {
                float v = (A == 0) ? k1_gray(u[e]) : __uint_as_float(u[e]);
                if constexpr (G::TEMPORAL) {
                    st[i][e] = k2_iir(st[i][e], v);
                    v = st[i][e];
                }
                pv[i][e] = v;
            }
        }
        if (f + 1 < f1) load(f + 1);  // the next frame's rows, in flight during this frame's spatial stages
        if constexpr (B <= 1 || A == 4) {
            // point groups: K1 alone, K1 K2, K2 alone, or K5 alone (on M')
#pragma unroll
            for (int i = 0; i < RW; ++i) emit(r0 + i, pv[i]);
        } else if constexpr (A <= 2) {
            // ---- K3 (then K4, K5) with the rows of the whole tile from shared memory
#pragma unroll
            for (int i = 0; i < RW; ++i) ys[r0 + i][lane] = make_float4(pv[i][0], pv[i][1], pv[i][2], pv[i][3]);
            __syncthreads();
            // rows streamed top to bottom: G' of row q as soon as hy of row q+1 exists
            float hy[3][C4];  // hy of rows q-1, q, q+1 (rolling)
#pragma unroll
            for (int i = 0; i < RW + 2; ++i) {
                const int r = r0 - 1 + i;
#pragma unroll
                for (int e = 0; e < C4; ++e) { hy[0][e] = hy[1][e]; hy[1][e] = hy[2][e]; }
                if (r >= 0 && r < TS) h121(ys[r][lane], hy[2]);  // warp-uniform
                const int q = r - 1;
                if (i < 2 || q < 1 || q > TS - 2) continue;
                float g[C4];
#pragma unroll
                for (int e = 0; e < C4; ++e) g[e] = tap121(hy[0][e], hy[1][e], hy[2][e]);
                if constexpr (B == 2) {
                    emit(q, g);
                } else {
                    if (edge_tile) {  // out-of-frame columns of G' take the edge column's value
                        if (xt < 0) {
                            const int sl = (0 - xt) / C4, se = (0 - xt) % C4;
                            const float ev = __shfl_sync(FULLM, se == 0 ? g[0] : se == 1 ? g[1] : se == 2 ? g[2] : g[3], sl);
#pragma unroll
                            for (int e = 0; e < C4; ++e) if (x0 + e < 0) g[e] = ev;
                        }
                        if (xt + TX > W) {
                            const int sl = (W - 1 - xt) / C4, se = (W - 1 - xt) % C4;
                            const float ev = __shfl_sync(FULLM, se == 0 ? g[0] : se == 1 ? g[1] : se == 2 ? g[2] : g[3], sl);
#pragma unroll
                            for (int e = 0; e < C4; ++e) if (x0 + e >= W) g[e] = ev;
                        }
                    }
                    gs[q][lane] = make_float4(g[0], g[1], g[2], g[3]);
                }
            }
            if constexpr (B >= 3) {
                __syncthreads();
            }
        } else {  // A == 3: K4 (+ K5) on the loaded G' rows
#pragma unroll
            for (int i = 0; i < RW; ++i) gs[r0 + i][lane] = make_float4(pv[i][0], pv[i][1], pv[i][2], pv[i][3]);
            __syncthreads();
        }
        if constexpr (G::H3) {
            // ---- K4 (+ K5) on output rows 2..29 (1..30 when the group starts at K4)
            constexpr int lo = HALO, hi = TS - HALO;
            float Dv[3][C4], Sv[3][C4];  // rows o-1, o, o+1 (rolling)
#pragma unroll
            for (int i = 0; i < RW + 2; ++i) {
                const int r = r0 - 1 + i;
#pragma unroll
                for (int e = 0; e < C4; ++e) {
                    Dv[0][e] = Dv[1][e]; Dv[1][e] = Dv[2][e];
                    Sv[0][e] = Sv[1][e]; Sv[1][e] = Sv[2][e];
                }
                if (r >= lo - 1 && r <= hi) {  // warp-uniform
                    const float4 g = gs[r][lane];
                    const float gl = __shfl_up_sync(FULLM, g.w, 1), gr = __shfl_down_sync(FULLM, g.x, 1);
                    const float gv[C4 + 2] = {gl, g.x, g.y, g.z, g.w, gr};
#pragma unroll
                    for (int e = 0; e < C4; ++e) {
                        Dv[2][e] = gv[e + 2] - gv[e];
                        Sv[2][e] = tap121(gv[e], gv[e + 1], gv[e + 2]);
                    }
                }
                const int o = r - 1;
                if (i < 2 || o < lo || o >= hi) continue;
                // rows o-1, o+1; at the frame's first and last rows the row itself (clamp on G')
                float m[C4];
                if (rows_inside) {  // warp-uniform: tiles away from the frame's top and bottom
#pragma unroll
                    for (int e = 0; e < C4; ++e)
                        m[e] = fabsf(tap121(Dv[0][e], Dv[1][e], Dv[2][e])) + fabsf(Sv[2][e] - Sv[0][e]);
                } else {
                    const bool top = y0 + o - 1 < 0, bot = y0 + o + 1 > H - 1;
#pragma unroll
                    for (int e = 0; e < C4; ++e) {
                        const float dc = Dv[1][e], sc = Sv[1][e];
                        const float dm = top ? dc : Dv[0][e], dp = bot ? dc : Dv[2][e];
                        const float sm = top ? sc : Sv[0][e], sp = bot ? sc : Sv[2][e];
                        m[e] = fabsf(tap121(dm, dc, dp)) + fabsf(sp - sm);
                    }
                }
                emit(o, m);
            }
        }
        if constexpr (G::H4) {
            count = __reduce_add_sync(FULLM, count);
            __syncwarp();  // the lanes' shared-memory region sums are visible
            const int64_t slot = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * TW + w;
            int32_t *sl = p.slots + ((int64_t)f * NSLOT + (int)(slot % NSLOT)) * NCNT;
            if (lane == 0 && count) atomicAdd(sl, (int)count);
            if (lane < NREG) {
                int *a2 = acc[w][lane];
                if (a2[0]) {
                    atomicAdd(sl + 1 + 3 * lane + 0, a2[0]);
                    atomicAdd(sl + 1 + 3 * lane + 1, a2[1]);
                    atomicAdd(sl + 1 + 3 * lane + 2, a2[2]);
                    a2[0] = a2[1] = a2[2] = 0;
                }
            }
            __syncwarp();
        }
        // before the next frame rewrites ys (read by K3 above when no second barrier follows
        // K3) or gs (written from the input rows when the group starts at K4)
        if constexpr ((G::H2 && B == 2) || A == 3) __syncthreads();
    }
}

// ---- the IIR recursion cut into chunks of CHUNK frames, so that chunks run in parallel.
// The filter is linear: started from state s before frame t0, y_{t0+j} = (1 - ALPHA)^(j+1) s
// + l_{t0+j}, where l is the same recursion started from 0. (1) Per chunk and pixel, l at
// the chunk's last frame; (2) per pixel, in chunk order, the state before each chunk:
// s_0 = Y_0 (so that y_0 = Y_0), s_k = (1 - ALPHA)^CHUNK s_{k-1} + l_end(k-1); (3) every
// group holding K2 runs each chunk from its s_k. The states are one FP32 plane per chunk;
// pass (2) overwrites l_end(k-1) with s_{k-1} in place.
constexpr int LW = 4, LR = TS / LW;  // local pass: warps per block, rows per warp (1 column per lane)

template <int A0>  // 0: RGBA frames, 1: Y' map
__global__ void __launch_bounds__(32 * LW) pc_iir_local_kernel(const PcParams p)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + lane;
    const int y = blockIdx.z * TS + LR * w;
    const int k = blockIdx.y;  // chunk (all but the last)
    if (x >= p.W) return;      // no block barriers here
    const int f0 = k * CHUNK;
    float l[LR];
#pragma unroll
    for (int i = 0; i < LR; ++i) l[i] = 0.0f;
    const uint32_t *base = p.in + x;
    const int nrows = min(LR, p.H - y);
#pragma unroll 4
    for (int f = f0; f < f0 + CHUNK; ++f) {  // unrolled: later frames' loads issue early
        const uint32_t *fr = base + (int64_t)f * p.in_fstride;
        uint32_t v[LR];
#pragma unroll
        for (int i = 0; i < LR; ++i) v[i] = i < nrows ? __ldg(fr + (int64_t)(y + i) * p.in_pitch) : 0u;
#pragma unroll
        for (int i = 0; i < LR; ++i) l[i] = k2_iir(l[i], A0 == 0 ? k1_gray(v[i]) : __uint_as_float(v[i]));
    }
    float *o = p.state + (int64_t)k * p.H * p.state_pitch + x;
#pragma unroll
    for (int i = 0; i < LR; ++i)
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
// The block stages KF_FRAMES frames of region sums in shared memory at a time (coalesced),
// so the walk's dependent chain never waits on a global load. The filter runs in FP32
// (stored as FP64): its chain of dependent operations per frame is the kernel's whole
// cost, and FP64 made it ten times longer on this part.
constexpr int KF_TRACKS = 32;  // tracks per block
constexpr int KF_FRAMES = 64;  // frames staged per round

__global__ void __launch_bounds__(KF_TRACKS) pc_kalman_kernel(const int32_t *regions, int T, int n, double *states,
                                                               int32_t *status)
{
    __shared__ int32_t zs[KF_FRAMES][KF_TRACKS][3];
    const int k0 = blockIdx.x * KF_TRACKS, k = k0 + threadIdx.x;
    const int nb = min(KF_TRACKS, n - k0);  // tracks of this block
    bool started = false;
    float px = 0, py = 0, vx = 0, vy = 0, P00 = 0, P01 = 0, P11 = 0;
    for (int t0 = 0; t0 < T; t0 += KF_FRAMES) {
        const int nt = min(KF_FRAMES, T - t0);
        __syncthreads();  // the previous round's values are consumed
        for (int i = threadIdx.x; i < nt * nb * 3; i += KF_TRACKS) {
            const int t = i / (nb * 3), j = i - t * nb * 3;
            zs[t][j / 3][j % 3] = regions[((int64_t)(t0 + t) * n + k0) * 3 + j];
        }
        __syncthreads();
        if (k >= n) continue;
        for (int t = 0; t < nt; ++t) {
            const int cnt = zs[t][threadIdx.x][0];
            const float inv_c = cnt > 0 ? 1.0f / (float)cnt : 0.0f;
            const float zx = (float)zs[t][threadIdx.x][1] * inv_c, zy = (float)zs[t][threadIdx.x][2] * inv_c;
            int s;
            if (!started) {
                if (cnt > 0) {
                    started = true;
                    px = zx;
                    py = zy;
                    vx = vy = 0.0f;
                    P00 = (float)KR;
                    P01 = 0.0f;
                    P11 = (float)KP0;
                    s = 1;
                } else {
                    s = 0;
                }
            } else {
                // predict: state by F, P by F P F' + Q with Q = q [[1/3, 1/2], [1/2, 1]]
                px += vx;
                py += vy;
                const float a = P00 + 2.0f * P01 + P11 + (float)(KQ / 3.0), b = P01 + P11 + (float)(KQ / 2.0), c = P11 + (float)KQ;
                P00 = a;
                P01 = b;
                P11 = c;
                if (cnt > 0) {
                    const float inv_s = 1.0f / (P00 + (float)KR), g0 = P00 * inv_s, g1 = P01 * inv_s;
                    const float ex = zx - px, ey = zy - py;
                    px += g0 * ex;
                    vx += g1 * ex;
                    py += g0 * ey;
                    vy += g1 * ey;
                    P11 -= g1 * P01;
                    P01 *= 1.0f - g0;
                    P00 *= 1.0f - g0;
                    s = 1;
                } else {
                    s = 2;
                }
            }
            double *o = states + ((int64_t)(t0 + t) * n + k) * 4;
            o[0] = px;
            o[1] = py;
            o[2] = vx;
            o[3] = vy;
            status[(int64_t)(t0 + t) * n + k] = s;
        }
    }
}

template <int A, int B>
int launch_one(const PcParams &p, cudaStream_t s)
{
    using G = Group<A, B>;
    const int64_t n_tiles = (int64_t)p.tiles_x * p.tiles_y;
    if constexpr (G::TEMPORAL) {
        // the chunk states first: local ends, then the carry (in place)
        const dim3 lg((unsigned)((p.W + 31) / 32), (unsigned)(p.n_chunks - 1), (unsigned)((p.H + TS - 1) / TS));
        if (p.n_chunks > 1) pc_iir_local_kernel<A><<<lg, 32 * LW, 0, s>>>(p);
        const int64_t px = (int64_t)p.W * p.H;
        pc_iir_carry_kernel<A><<<(unsigned)((px + 255) / 256), 256, 0, s>>>(p);
        pc_tile_kernel<A, B><<<dim3((unsigned)n_tiles, (unsigned)p.n_chunks), 32 * TW, 0, s>>>(p);
    } else {
        pc_tile_kernel<A, B><<<dim3((unsigned)n_tiles, (unsigned)p.T), 32 * TW, 0, s>>>(p);
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
    if (!v || !v->rgba || v->W <= 0 || v->H <= 0 || v->T < 0 || v->pitch < v->W || v->pitch % 4 || !aligned(v->rgba, 16))
        return KF_EINVAL;
    if (v->W > (1 << 24) || v->H > (1 << 24) || !kf::volume_ok(v->W, v->H, v->T) || v->W * v->H > 0x7fffffffLL)
        return KF_EINVAL;
    if (!sums_fit(v->W, v->H)) return KF_EINVAL;
    return KF_OK;
}
kf_status check_out(const kf_pc_out *o, int64_t W)
{
    if (!o || !o->mask || o->mask_pitch < W || o->mask_pitch % 4 || !aligned(o->mask, 16) || !o->counts || !o->regions ||
        !aligned(o->counts, 4) || !aligned(o->regions, 4))
        return KF_EINVAL;
    return KF_OK;
}

PcParams params_for(int a, int b, int64_t W, int64_t H, int64_t T)
{
    PcParams p{};
    const int halo = halo_of(a, b), hc = halo ? 4 : 0;
    const int outw = TX - 2 * hc, outh = TS - 2 * halo;
    p.W = (int)W;
    p.H = (int)H;
    p.T = (int)T;
    p.tiles_x = (int)((W + outw - 1) / outw);
    p.tiles_y = (int)((H + outh - 1) / outh);
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
    if (n_tiles > 0x7fffffffLL || (!temporal && T > 65535)) return KF_EINVAL;
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
            const int halo = halo_of(a, i), hc = halo ? 4 : 0;
            const double read_factor = (double)TX * TS / ((double)(TX - 2 * hc) * (TS - 2 * halo));
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
    if (!ctx || !bytes || !kf::volume_ok(W, H, T) || cuts >= 16) return KF_EINVAL;
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
    if (kf_pc_workspace_bytes(ctx, cuts, video->W, video->H, video->T, &need) != KF_OK) return KF_EINVAL;
    if (need && (!workspace || !aligned(workspace, 256))) return KF_EINVAL;
    if (workspace_bytes < need) return KF_ENOMEM;
    kf::DeviceScope dev_scope(dev);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
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
    if (!ctx || !bytes || a < 0 || b < a || b >= KF_PC_STAGES || !kf::volume_ok(W, H, T)) return KF_EINVAL;
    *bytes = (holds_iir(a, b) ? state_bytes(W, H, T) : 0) + (b == 4 ? slot_bytes(T) : 0);
    return KF_OK;
}

kf_status kf_pc_run_group(kf_ctx *ctx, int a, int b, const kf_pc_video *video, const float *in, int64_t in_pitch,
                          float *out, int64_t out_pitch, const kf_pc_out *out_mask, void *workspace,
                          size_t workspace_bytes, void *stream)
{
    if (!ctx || a < 0 || b < a || b >= KF_PC_STAGES) return KF_EINVAL;
    // geometry from the video descriptor (its rgba is only read when a == 0)
    if (!video || !kf::volume_ok(video->W, video->H, video->T) || !sums_fit(video->W, video->H))
        return KF_EINVAL;
    const int64_t W = video->W, H = video->H, T = video->T;
    if (a == 0) {
        const kf_status st = check_video(video);
        if (st != KF_OK) return st;
    } else if (!in || in_pitch < W || in_pitch % 4 || !aligned(in, 16)) {
        return KF_EINVAL;
    }
    if (b == 4) {
        const kf_status st = check_out(out_mask, W);
        if (st != KF_OK) return st;
    } else if (!out || out_pitch < W || out_pitch % 4 || !aligned(out, 16)) {
        return KF_EINVAL;
    }
    const size_t need = (holds_iir(a, b) ? state_bytes(W, H, T) : 0) + (b == 4 ? slot_bytes(T) : 0);
    if (need) {
        if (!workspace || !aligned(workspace, 256)) return KF_EINVAL;
        if (workspace_bytes < need) return KF_ENOMEM;
    }
    const int dev = kf::ctx_device(ctx);
    if (dev < 0) return KF_ESTATE;
    kf::DeviceScope dev_scope(dev);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
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
    kf::DeviceScope dev_scope(dev);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
    pc_kalman_kernel<<<(n_tracks + KF_TRACKS - 1) / KF_TRACKS, KF_TRACKS, 0, static_cast<cudaStream_t>(stream)>>>(
        regions, (int)T, n_tracks, states, status);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : fail(ctx, (int)e);
}

}  // extern "C"
