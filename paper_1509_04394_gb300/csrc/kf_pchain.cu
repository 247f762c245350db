// kf_pchain.cu -- the paper's own chain (Table II / Table IV): K1 convert RGBA to gray,
// K2 IIR filter, K3 Gaussian smoothing, K4 gradient filter, K5 threshold computation,
// any contiguous group of them fused into one kernel (Sec. V-B, Eq. 2), and K6, the
// Kalman filter over feature positions, after the kernel-to-kernel dependency.
//
// Group kernel pc_kernel<A, B> (0-based stages A..B). Each warp owns a 32 x 32 tile of
// the group's input: lane = column, the 32 rows streamed top to bottom in registers.
// Horizontal taps are warp shuffles, vertical taps a few rows of registers; a group with
// K3 and K4 has a 2-pixel halo and writes the inner 28 x 28 (30 x 30 with one of them).
// A group holding K2 (the IIR filter, a recursion over frames) keeps the filter state of
// its 32 rows per lane in registers and walks every frame of the video in order, loading
// the next frame's tile while it computes the current one; no filter state goes through
// memory. Other groups run one (tile, frame) per warp.
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

struct PcParams {
    const uint32_t *in;   // RGBA pixels (A == 0) or FP32 bit patterns
    int64_t in_pitch, in_fstride;    // elements
    void *out;            // FP32 map (B < 4) or u8 mask (B == 4)
    int64_t out_pitch, out_fstride;  // elements
    int W, H, T;
    int tiles_x, tiles_y;
    int32_t *counts, *regions;       // B == 4
};

// ---- the stages (one definition each, used by every group)
__device__ __forceinline__ float k1_gray(uint32_t rgba)
{
    const float r = (float)(rgba & 0xffu), g = (float)((rgba >> 8) & 0xffu), b = (float)((rgba >> 16) & 0xffu);
    return fmaf(29.0f, b, fmaf(150.0f, g, 77.0f * r));  // integer <= 65280: exact
}
__device__ __forceinline__ float k2_iir(float prev, float Y, bool first) { return first ? Y : fmaf(ALPHA, Y - prev, prev); }
// [1 2 1] of three neighbours (the centre weighted 2)
__device__ __forceinline__ float tap121(float l, float c, float r) { return fmaf(2.0f, c, l + r); }

template <int A, int B> struct Group {
    static constexpr bool H1 = A <= 1 && 1 <= B, H2 = A <= 2 && 2 <= B, H3 = A <= 3 && 3 <= B, H4 = B == 4;
    static constexpr int HALO = (H2 ? 1 : 0) + (H3 ? 1 : 0);
    static constexpr int OUT = TS - 2 * HALO;  // output tile side
    static constexpr bool TEMPORAL = H1;
};

template <int A, int B>
__global__ void __launch_bounds__(32 * WPB) pc_kernel(const PcParams p)
{
    using G = Group<A, B>;
    constexpr int HALO = G::HALO, OUT = G::OUT;
    __shared__ int acc[WPB][NREG][3];  // this frame's region sums of the warp (B == 4)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    const int64_t n_tiles = (int64_t)p.tiles_x * p.tiles_y;
    int64_t tile;
    int f_begin, f_end;
    if constexpr (G::TEMPORAL) {
        if (gw >= n_tiles) return;  // warp-uniform; no block barriers below
        tile = gw;
        f_begin = 0;
        f_end = p.T;
    } else {
        if (gw >= n_tiles * p.T) return;
        tile = gw % n_tiles;
        f_begin = (int)(gw / n_tiles);
        f_end = f_begin + 1;
    }
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
    [[maybe_unused]] float st[TS];  // IIR state of each row (TEMPORAL)
    load(f_begin, buf);

    for (int f = f_begin; f < f_end; ++f) {
        uint32_t cur[TS];
#pragma unroll
        for (int r = 0; r < TS; ++r) cur[r] = buf[r];
        if (f + 1 < f_end) load(f + 1, buf);  // in flight while this frame computes
        const bool first = f == 0;
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
            if constexpr (A <= 2) {
                // ---- K1, K2
                float yv;
                if constexpr (A == 0) {
                    const float Y = k1_gray(v);
                    if constexpr (B == 0) { emit(r, Y); continue; }
                    yv = k2_iir(st[r], Y, first);
                    st[r] = yv;
                } else if constexpr (A == 1) {
                    yv = k2_iir(st[r], __uint_as_float(v), first);
                    st[r] = yv;
                } else {
                    yv = __uint_as_float(v);
                }
                if constexpr (B == 1) { emit(r, yv); continue; }
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
            if (lane == 0 && count) atomicAdd(p.counts + f, (int)count);
            if (lane < NREG) {
                int *a = acc[wib][lane];
                if (a[0]) {
                    int32_t *g = p.regions + ((int64_t)f * NREG + lane) * 3;
                    atomicAdd(g + 0, a[0]);
                    atomicAdd(g + 1, a[1]);
                    atomicAdd(g + 2, a[2]);
                    a[0] = a[1] = a[2] = 0;
                }
            }
            __syncwarp();
        }
    }
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
        // one warp per block: the few long-lived warps spread over every SM
        pc_kernel<A, B><<<(unsigned)n_tiles, 32, 0, s>>>(p);
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

// one group over prepared pointers; zeroes counts and regions first when it ends at K5
kf_status run_group(kf_ctx *ctx, int a, int b, const uint32_t *in, int64_t in_pitch, void *out, int64_t out_pitch,
                    int64_t W, int64_t H, int64_t T, int32_t *counts, int32_t *regions, cudaStream_t s)
{
    if (T == 0) return KF_OK;
    PcParams p = params_for(a, b, W, H, T);
    p.in = in;
    p.in_pitch = in_pitch;
    p.in_fstride = in_pitch * H;
    p.out = out;
    p.out_pitch = out_pitch;
    p.out_fstride = out_pitch * H;
    p.counts = counts;
    p.regions = regions;
    if (b == 4) {
        cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)T, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(regions, 0, sizeof(int32_t) * 3 * NREG * (size_t)T, s);
        if (e != cudaSuccess) return fail(ctx, (int)e);
    }
    const int64_t n_tiles = (int64_t)p.tiles_x * p.tiles_y;
    const bool temporal = a <= 1 && 1 <= b;
    if ((temporal ? n_tiles : (n_tiles * T + WPB - 1) / WPB) > 0x7fffffffLL) return KF_EINVAL;
    const int e = launch_group(a, b, p, s);
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
    *bytes = n_cuts == 0 ? 0 : (n_cuts == 1 ? plane_a : 2 * plane_a);
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
    float *planes[2] = {static_cast<float *>(workspace),
                        workspace ? reinterpret_cast<float *>(static_cast<char *>(workspace) + plane_a) : nullptr};
    const uint32_t *in = reinterpret_cast<const uint32_t *>(video->rgba);
    int64_t in_pitch = video->pitch;
    int a = 0, k = 0;
    for (int i = 0; i < KF_PC_STAGES; ++i) {
        if (i != KF_PC_STAGES - 1 && !(cuts >> i & 1)) continue;
        const bool last = i == KF_PC_STAGES - 1;
        void *o = last ? static_cast<void *>(out->mask) : static_cast<void *>(planes[k % 2]);
        const int64_t op = last ? out->mask_pitch : wp;
        st = run_group(ctx, a, i, in, in_pitch, o, op, W, H, T, out->counts, out->regions, s);
        if (st != KF_OK) return st;
        in = reinterpret_cast<const uint32_t *>(planes[k % 2]);
        in_pitch = wp;
        ++k;
        a = i + 1;
    }
    return KF_OK;
}

kf_status kf_pc_run_group(kf_ctx *ctx, int a, int b, const kf_pc_video *video, const float *in, int64_t in_pitch,
                          float *out, int64_t out_pitch, const kf_pc_out *out_mask, void *stream)
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
    const int dev = kf::ctx_device(ctx);
    if (dev < 0) return KF_ESTATE;
    if (cudaSetDevice(dev) != cudaSuccess) return KF_ECUDA;
    const uint32_t *src = a == 0 ? reinterpret_cast<const uint32_t *>(video->rgba) : reinterpret_cast<const uint32_t *>(in);
    const int64_t sp = a == 0 ? video->pitch : in_pitch;
    void *dst = b == 4 ? static_cast<void *>(out_mask->mask) : static_cast<void *>(out);
    const int64_t dp = b == 4 ? out_mask->mask_pitch : out_pitch;
    return run_group(ctx, a, b, src, sp, dst, dp, W, H, T, b == 4 ? out_mask->counts : nullptr,
                     b == 4 ? out_mask->regions : nullptr, static_cast<cudaStream_t>(stream));
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
