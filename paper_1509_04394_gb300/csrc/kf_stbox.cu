// kf_stbox.cu -- a spatio-temporal fused group run over x * x * t boxes (Sec. VI-C to
// VI-E: Alg. 2's input box, Eq. 3's data utilisation, Eq. 5 / Eq. 6's box shape).
//
// The group: K1 RGBA to gray, Kt the temporal binomial over the current and the n
// previous frames (n = 1, 2 or 4), K3 3x3 binomial smoothing, K4 Sobel L1 magnitude, K5
// threshold with per-frame counts. One-sided reaches: dx = 2, dt = n. Every map is an
// integer multiple of a fixed scale (gray 77 R + 150 G + 29 B, temporal weights C(n, k),
// smoothing weights (1,2,1)x(1,2,1), unnormalised Sobel), so the chain is computed
// exactly in 32-bit integers and M > 0.25 is M_int > 261120 * 2^n.
//
// One block per box. The box's frames stream through shared memory in time order: a TMA
// copy brings the (x + 8) x (x + 4) RGBA pixels of the next frame (the box with its
// two-pixel spatial halo, widened to 16-byte column boundaries) into a staging plane while
// the block computes the current frame; the block turns it into a 16-bit gray plane in a
// ring of n + 1 planes. So the temporal halo -- the n frames before the current one -- stays
// on chip for the whole box and each input frame of the box is read once: a box reads
// (x + 4)^2 (t + n) pixels (plus the column widening) and writes x^2 t mask bytes.
// Per frame, pass B forms the smoothed map G over (x + 2) x (x + 4) from the ring (4
// columns per thread, a 3-row vertical window in registers), pass C the Sobel magnitude,
// threshold and mask stores over x * x (4 columns per thread, 4 mask bytes per store).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include "kf_ctx.h"

namespace kf {
namespace {

constexpr unsigned ST_WAIT_LIMIT = 1u << 22;  // try_wait rounds before giving up
constexpr int ST_DEVERR_TIMEOUT = 1;
constexpr int ST_MAX_SMEM = 227 * 1024;

struct StParams {
    CUtensorMap tmap;  // RGBA frames as 32-bit elements {W, H, T}; box {x + 8, x + 4, 1}
    uint8_t *mask;
    int64_t mask_pitch, mask_fstride;
    int32_t *counts;
    int *err;
    int W, H, T;
    int x, t;              // box: x * x pixels, t frames
    int boxes_x, boxes_y;  // boxes per frame row / column
    int seg;               // rows per work item of passes B and C
    int thr_shift;         // n
    // shared memory layout (bytes from the 128-aligned base)
    int off_ring, off_g, off_bar;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity)
{
    for (unsigned i = 0; i < ST_WAIT_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_frame(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t gray_of(uint32_t rgba)
{
    return 77u * (rgba & 0xffu) + 150u * ((rgba >> 8) & 0xffu) + 29u * ((rgba >> 16) & 0xffu);
}

// binomial weight C(N, k)
template <int N> __device__ __forceinline__ int binom(int k);
template <> __device__ __forceinline__ int binom<1>(int) { return 1; }
template <> __device__ __forceinline__ int binom<2>(int k) { return k == 1 ? 2 : 1; }
template <> __device__ __forceinline__ int binom<4>(int k) { return k == 2 ? 6 : (k == 1 || k == 3) ? 4 : 1; }

template <int N>
__global__ void __launch_bounds__(256) st_box_kernel(const __grid_constant__ StParams p)
{
    extern __shared__ __align__(128) unsigned char st_smem[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)st_smem + 127) & ~(uintptr_t)127);
    const int x = p.x, SR = x + 4, SC = x + 8;  // staging / ring plane: rows, columns
    const uint32_t *stage = reinterpret_cast<const uint32_t *>(base);
    uint16_t *ring = reinterpret_cast<uint16_t *>(base + p.off_ring);
    int32_t *G = reinterpret_cast<int32_t *>(base + p.off_g);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + p.off_bar);
    const int GW = x + 4;           // G plane columns (x + 2 used)
    const int plane = SR * SC;      // u16 elements per ring plane

    const int b = blockIdx.x;
    const int nb_xy = p.boxes_x * p.boxes_y;
    const int bt = b / nb_xy, bxy = b - bt * nb_xy;
    const int by = bxy / p.boxes_x, bx = bxy - by * p.boxes_x;
    const int x0 = bx * x, y0 = by * x, t0 = bt * p.t;
    const int t_end = min(t0 + p.t, p.T);
    const int n_planes = t_end - (t0 - N);  // the n frames before the box, then its own
    const int tid = threadIdx.x;
    const unsigned stage_bytes = (unsigned)(SR * SC * 4);

    if (tid == 0) {
        bar_init(bar);
        bar_expect(bar, stage_bytes);
        tma_frame(base, &p.tmap, x0 - 4, y0 - 2, max(t0 - N, 0), bar);
    }
    __syncthreads();

    // staging index of a clamped image coordinate (the clamped pixel always lies in the box)
    const bool inner_x = x0 - 4 >= 0 && x0 + x + 4 <= p.W;
    const bool inner_y = y0 - 2 >= 0 && y0 + x + 2 <= p.H;
    const int thr = 261120 << p.thr_shift;
    const int gcols = GW / 4, ocols = x / 4;
    const int segs_b = (x + 2 + p.seg - 1) / p.seg, segs_c = (x + p.seg - 1) / p.seg;

    for (int pl = 0; pl < n_planes; ++pl) {
        const bool ok = bar_wait(bar, (unsigned)(pl & 1));
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicOr(p.err, ST_DEVERR_TIMEOUT);
                bar_wait(bar, (unsigned)(pl & 1));  // the copy in flight, once more (bounded)
            }
            return;
        }
        // the staged frame -> gray ring slot pl % (N + 1), two pixels per step
        uint16_t *slot = ring + (pl % (N + 1)) * plane;
        for (int i = tid; i < SR * (SC / 2); i += blockDim.x) {
            const int r = i / (SC / 2), c = 2 * (i - r * (SC / 2));
            uint32_t a, bb;
            if (inner_x && inner_y) {
                const uint2 w = *reinterpret_cast<const uint2 *>(stage + r * SC + c);
                a = w.x;
                bb = w.y;
            } else {
                const int ry = min(max(y0 - 2 + r, 0), p.H - 1) - (y0 - 2);
                const int ca = min(max(x0 - 4 + c, 0), p.W - 1) - (x0 - 4);
                const int cb = min(max(x0 - 3 + c, 0), p.W - 1) - (x0 - 4);
                a = stage[ry * SC + ca];
                bb = stage[ry * SC + cb];
            }
            *reinterpret_cast<uint32_t *>(slot + r * SC + c) = gray_of(a) | (gray_of(bb) << 16);
        }
        __syncthreads();
        if (tid == 0 && pl + 1 < n_planes) {
            bar_expect(bar, stage_bytes);
            tma_frame(base, &p.tmap, x0 - 4, y0 - 2, max(t0 - N + pl + 1, 0), bar);
        }
        if (pl < N) continue;  // a frame of the temporal halo only
        const int f = t0 - N + pl;

        // pass B: G over rows 0..x+1 (image y0-1..), columns 0..x+3 (image x0-1..)
        for (int it = tid; it < gcols * segs_b; it += blockDim.x) {
            const int g = 4 * (it % gcols), r0 = (it / gcols) * p.seg, r1 = min(r0 + p.seg, x + 2);
            int hm2[4] = {0, 0, 0, 0}, hm1[4] = {0, 0, 0, 0};
            for (int i = r0; i < r1 + 2; ++i) {  // ring rows i (image y0-2+i)
                int z[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) z[j] = 0;
#pragma unroll
                for (int k = 0; k <= N; ++k) {
                    const uint16_t *row = ring + ((pl - N + k) % (N + 1)) * plane + i * SC + g + 2;
                    const uint32_t *w = reinterpret_cast<const uint32_t *>(row);
                    const int wk = binom<N>(k);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const uint32_t v = w[j];
                        z[2 * j] += wk * (int)(v & 0xffffu);
                        z[2 * j + 1] += wk * (int)(v >> 16);
                    }
                }
                int h[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) h[c] = z[c] + 2 * z[c + 1] + z[c + 2];
                if (i >= r0 + 2) {
                    int4 o;
                    o.x = hm2[0] + 2 * hm1[0] + h[0];
                    o.y = hm2[1] + 2 * hm1[1] + h[1];
                    o.z = hm2[2] + 2 * hm1[2] + h[2];
                    o.w = hm2[3] + 2 * hm1[3] + h[3];
                    *reinterpret_cast<int4 *>(G + (i - 2) * GW + g) = o;
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    hm2[c] = hm1[c];
                    hm1[c] = h[c];
                }
            }
        }
        __syncthreads();

        // pass C: Sobel magnitude, threshold, mask and count over the box's x * x outputs
        int count = 0;
        uint8_t *mframe = p.mask + (int64_t)f * p.mask_fstride;
        for (int it = tid; it < ocols * segs_c; it += blockDim.x) {
            const int o = 4 * (it % ocols), r0 = (it / ocols) * p.seg, r1 = min(r0 + p.seg, x);
            int dxm2[4] = {0, 0, 0, 0}, dxm1[4] = {0, 0, 0, 0}, sxm2[4] = {0, 0, 0, 0}, sxm1[4] = {0, 0, 0, 0};
            for (int gr = r0; gr < r1 + 2; ++gr) {  // G rows gr (output row gr - 1 centre)
                const int4 a = *reinterpret_cast<const int4 *>(G + gr * GW + o);
                const int2 c2 = *reinterpret_cast<const int2 *>(G + gr * GW + o + 4);
                const int v[6] = {a.x, a.y, a.z, a.w, c2.x, c2.y};
                int dx[4], sx[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    dx[c] = v[c + 2] - v[c];
                    sx[c] = v[c] + 2 * v[c + 1] + v[c + 2];
                }
                if (gr >= r0 + 2) {
                    const int r = gr - 2;  // output row (image y0 + r)
                    uint32_t bits = 0;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int gx = dxm2[c] + 2 * dxm1[c] + dx[c];
                        const int gy = sx[c] - sxm2[c];
                        bits |= (uint32_t)(abs(gx) + abs(gy) > thr) << (8 * c);
                    }
                    const int yy = y0 + r, xx = x0 + o;
                    if (yy < p.H && xx < p.W) {
                        uint8_t *dst = mframe + (int64_t)yy * p.mask_pitch + xx;
                        if (xx + 4 <= p.W) {
                            *reinterpret_cast<uint32_t *>(dst) = bits;
                        } else {
                            bits &= (1u << (8 * (p.W - xx))) - 1u;
                            for (int c = 0; c < p.W - xx; ++c) dst[c] = (uint8_t)(bits >> (8 * c));
                        }
                        count += __popc(bits);
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    dxm2[c] = dxm1[c];
                    dxm1[c] = dx[c];
                    sxm2[c] = sxm1[c];
                    sxm1[c] = sx[c];
                }
            }
        }
        count = __reduce_add_sync(0xffffffffu, count);
        if ((tid & 31) == 0 && count) atomicAdd(p.counts + f, count);
    }
}

// shared memory plan of a box side and temporal reach
struct StSmem {
    int off_ring, off_g, off_bar, total;
};
StSmem st_plan(int x, int n)
{
    auto up = [](int v, int a) { return (v + a - 1) / a * a; };
    StSmem s;
    const int SR = x + 4, SC = x + 8;
    s.off_ring = up(SR * SC * 4, 128);
    s.off_g = up(s.off_ring + (n + 1) * SR * SC * 2, 128);
    s.off_bar = up(s.off_g + (x + 2) * (x + 4) * 4, 128);
    s.total = s.off_bar + 8 + 128;  // + alignment slack of the dynamic base
    return s;
}

bool valid_n(int n) { return n == 1 || n == 2 || n == 4; }

}  // namespace

// launch configuration of a box: threads and rows per work item
void st_config(int x, int *threads, int *seg)
{
    int th = (x * x / 32 + 31) / 32 * 32;
    th = th < 32 ? 32 : (th > 256 ? 256 : th);
    int s = (x * (x / 4) + th - 1) / th;
    *threads = th;
    *seg = s < 2 ? 2 : s;
}

}  // namespace kf

using kf::StParams;

namespace {
PFN_cuTensorMapEncodeTiled_v12000 st_encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

kf_status st_fail(kf_ctx *c, cudaError_t e)
{
    c->last_cuda = (int)e;
    return KF_ECUDA;
}
}  // namespace

extern "C" {

kf_status kf_st_smem_bytes(int n, int x, size_t *bytes)
{
    if (!bytes || !kf::valid_n(n) || x < 8 || x > 248 || x % 8) return KF_EINVAL;
    *bytes = (size_t)kf::st_plan(x, n).total;
    return KF_OK;
}

kf_status kf_st_traffic(int64_t W, int64_t H, int64_t T, int x, int t, int n, double *model_bytes, double *clipped_bytes)
{
    if (W < 1 || H < 1 || T < 0 || x < 1 || t < 1 || !kf::valid_n(n)) return KF_EINVAL;
    const double B = (double)W * (double)H * (double)T / ((double)x * x * t);
    const double in = (double)(x + 4) * (x + 4) * (t + n);
    if (model_bytes) *model_bytes = B * (4.0 * in + (double)x * x * t);
    if (clipped_bytes) {
        // sum over the tiling of each box's input extent clipped to the volume: separable
        auto span = [](int64_t N, int64_t b, int64_t lo, int64_t hi) {
            double s = 0;
            for (int64_t v = 0; v < N; v += b) {
                const int64_t a = v - lo < 0 ? 0 : v - lo, e = v + b + hi > N ? N : v + b + hi;
                s += (double)(e - a);
            }
            return s;
        };
        *clipped_bytes = 4.0 * span(W, x, 2, 2) * span(H, x, 2, 2) * span(T, t, n, 0) + (double)W * H * T;
    }
    return KF_OK;
}

kf_status kf_st_box_eq6(double beta, int n, double *x, double *t)
{
    if (!(beta > 0) || !kf::valid_n(n) || !x || !t) return KF_EINVAL;
    const double dx = 2.0, dt = (double)n;
    *x = cbrt(2.0 * beta * dx / dt);
    *t = beta / (*x * *x);
    return KF_OK;
}

kf_status kf_st_run(kf_ctx *ctx, const kf_pc_video *video, uint8_t *mask, int64_t mask_pitch, int32_t *counts, int n,
                    int x, int t, void *stream)
{
    if (!ctx || !video || !kf::valid_n(n) || x < 8 || x % 8 || t < 1) return KF_EINVAL;
    const int64_t W = video->W, H = video->H, T = video->T;
    if (W < 1 || H < 1 || T < 0 || W > 0x7fffffff || H > 0x7fffffff || T > 0x7fffffff) return KF_EINVAL;
    if (T == 0) return KF_OK;
    if (!video->rgba || !mask || !counts || (uintptr_t)video->rgba % 16 || (uintptr_t)mask % 16) return KF_EINVAL;
    if (video->pitch < W || video->pitch % 4 || mask_pitch < W || mask_pitch % 4) return KF_EINVAL;
    const kf::StSmem sm = kf::st_plan(x, n);
    if (sm.total > kf::ST_MAX_SMEM) return KF_EINVAL;
    const int64_t bxn = (W + x - 1) / x, byn = (H + x - 1) / x, btn = (T + t - 1) / t;
    if (bxn * byn * btn > 0x7fffffff) return KF_EINVAL;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return st_fail(ctx, e);

    StParams p{};
    PFN_cuTensorMapEncodeTiled_v12000 fn = st_encode_fn();
    if (!fn) return KF_EINVAL;
    cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
    cuuint64_t strides[2] = {(cuuint64_t)(video->pitch * 4), (cuuint64_t)(video->pitch * H * 4)};
    cuuint32_t box[3] = {(cuuint32_t)(x + 8), (cuuint32_t)(x + 4), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&p.tmap, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint8_t *>(video->rgba), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return KF_EINVAL;
    p.mask = mask;
    p.mask_pitch = mask_pitch;
    p.mask_fstride = mask_pitch * H;
    p.counts = counts;
    p.err = ctx->d_err;
    p.W = (int)W;
    p.H = (int)H;
    p.T = (int)T;
    p.x = x;
    p.t = t;
    p.boxes_x = (int)bxn;
    p.boxes_y = (int)byn;
    p.thr_shift = n;
    p.off_ring = sm.off_ring;
    p.off_g = sm.off_g;
    p.off_bar = sm.off_bar;
    int threads = 0;
    kf::st_config(x, &threads, &p.seg);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)T, s);
    if (e != cudaSuccess) return st_fail(ctx, e);
    void (*kern)(StParams) = n == 1 ? kf::st_box_kernel<1> : (n == 2 ? kf::st_box_kernel<2> : kf::st_box_kernel<4>);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, sm.total);
    if (e != cudaSuccess) return st_fail(ctx, e);
    kern<<<(unsigned)(bxn * byn * btn), threads, sm.total, s>>>(p);
    e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : st_fail(ctx, e);
}

}  // extern "C"
