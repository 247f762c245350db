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
// One block per box, the box side X a compile-time constant. The box's frames stream
// through shared memory in time order: a TMA copy brings the (X + 8) x (X + 4) RGBA pixels
// of the next frame (the box with its two-pixel spatial halo, widened to 16-byte column
// boundaries) into a staging plane while the block computes the current frame. Each
// thread converts the same pixel pairs in every frame, so the gray values of the n
// previous frames -- the temporal halo -- stay on chip for the whole box in a ring only
// that thread touches, and each input frame of the box is read once: a box reads
// (X + 4)^2 (t + n) pixels (plus the column widening) and writes X^2 t mask bytes.
// Per frame: K1 + Kt write the temporal map Z; pass B forms the smoothed map G over
// (X + 2) x (X + 4) (4 columns per thread, a 3-row vertical window in registers); pass C
// the Sobel magnitude, threshold and mask stores over X * X (4 columns per thread, 4 mask
// bytes per store).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include "kf_ctx.h"
#include "kf_device.h"

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
    int t;                 // box depth in frames (the side is the kernel's X)
    int boxes_x, boxes_y;  // boxes per frame row / column
    unsigned wait_polls;   // try_wait rounds of the wait for a frame's copy (the drain after an
                           // expired wait always gets ST_WAIT_LIMIT)
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
__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity, unsigned polls = ST_WAIT_LIMIT)
{
    for (unsigned i = 0; i < polls; ++i) {
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

// K1 for two RGBA pixels at once: the R, G and B bytes of both gathered into 16-bit
// halves by byte permutes, so one multiply-add chain gives both gray values (each at
// most 65280, so the halves never carry into each other): lo = gray(a), hi = gray(b).
__device__ __forceinline__ uint32_t gray_pair(uint32_t a, uint32_t b)
{
    const uint32_t u = __byte_perm(a, b, 0x5140);  // a.R, b.R, a.G, b.G
    const uint32_t v = __byte_perm(a, b, 0x0062);  // a.B, b.B
    const uint32_t r = __byte_perm(u, 0u, 0x4140), g = __byte_perm(u, 0u, 0x4342), bl = __byte_perm(v, 0u, 0x4140);
    return 77u * r + 150u * g + 29u * bl;
}

// binomial weight C(N, k)
template <int N> __host__ __device__ constexpr int binom(int k)
{
    return N == 1 ? 1 : N == 2 ? (k == 1 ? 2 : 1) : (k == 2 ? 6 : (k == 1 || k == 3) ? 4 : 1);
}

// Launch shape of a box side X: threads per block (about ten pixel pairs of a staged
// frame per thread) and rows per work item of passes B and C.
template <int X> struct BoxCfg {
    static constexpr int THREADS = X <= 16 ? 32 : X <= 32 ? 64 : X <= 48 ? 128 : X <= 64 ? 256 : 512;
    // rows per work item: as many items as threads, about, in each pass
    static constexpr int SEG_B = (X + 2 + THREADS / ((X + 4) / 4) - 1) / (THREADS / ((X + 4) / 4));
    static constexpr int SEG_C = (X + THREADS / (X / 4) - 1) / (THREADS / (X / 4));
    // row loops of passes B and C fully unrolled (compile-time register windows) where the
    // register budget allows it without spilling; measured 15 % faster at X = 64
    static constexpr int UNROLL_B = X >= 32 && X <= 64 ? SEG_B + 2 : 1;
    static constexpr int UNROLL_C = X >= 32 && X <= 64 ? SEG_C + 2 : 1;
    static constexpr int SR = X + 4, SC = X + 8, GW = X + 4;  // staged rows / columns; G columns
    static constexpr int PAIRS = SR * (SC / 2);                 // pixel pairs of a staged frame
    static constexpr int STAGE_BYTES = SR * SC * 4;
    __host__ __device__ static constexpr int up(int v) { return (v + 127) / 128 * 128; }
    static constexpr int OFF_Z = up(STAGE_BYTES);
    static constexpr int OFF_G = OFF_Z + up(SR * SC * 4);
    static constexpr int OFF_RING = OFF_G + up((X + 2) * GW * 4);
    template <int N> __host__ __device__ static constexpr int off_bar() { return OFF_RING + up(N * PAIRS * 4); }
    template <int N> __host__ __device__ static constexpr int smem() { return off_bar<N>() + 8 + 128; }  // + base alignment slack
};

// Per-box constants shared by the passes.
struct BoxPos {
    int x0, y0;          // the box's first column / row
    bool inner;          // the staged frame needs no clamping
    int gr_lo, gr_hi;    // G plane rows inside the frame (G row j is image row y0-1+j)
    int g_lo, g_hi;      // G plane columns inside the frame (G column j is image column x0-1+j)
};

// K1 + Kt: the staged frame (pl-th plane of the box) -> gray pairs -> the temporal binomial
// into Z (output planes only); the thread's ring keeps the gray of its pairs' last N frames.
template <int N, int X>
__device__ __forceinline__ void convert_frame(const StParams &p, const BoxPos &b, const uint32_t *stage, uint32_t *ring,
                                              int32_t *Z, int pl)
{
    using C = BoxCfg<X>;
    constexpr int SC = C::SC;
    const bool out_frame = pl >= N;
    const int slot0 = pl % N;  // the ring slot of plane pl - N, overwritten by plane pl
    // pair i = threadIdx.x + k THREADS sits at row r, column c; walked without divisions
    constexpr int PR = SC / 2, R_STEP = C::THREADS / PR, C_STEP = 2 * (C::THREADS - R_STEP * PR);
    int r = threadIdx.x / PR, c = 2 * (threadIdx.x - r * PR);
#pragma unroll 2
    for (int i = threadIdx.x; i < C::PAIRS; i += C::THREADS) {
        uint32_t a, bb;
        if (b.inner) {
            const uint2 w = *reinterpret_cast<const uint2 *>(stage + r * SC + c);
            a = w.x;
            bb = w.y;
        } else {
            const int ry = min(max(b.y0 - 2 + r, 0), p.H - 1) - (b.y0 - 2);
            const int ca = min(max(b.x0 - 4 + c, 0), p.W - 1) - (b.x0 - 4);
            const int cb = min(max(b.x0 - 3 + c, 0), p.W - 1) - (b.x0 - 4);
            a = stage[ry * SC + ca];
            bb = stage[ry * SC + cb];
        }
        const uint32_t g = gray_pair(a, bb);
        if (out_frame) {
            int lo = (int)(g & 0xffffu), hi = (int)(g >> 16);
#pragma unroll
            for (int k = 0; k < N; ++k) {  // plane pl - N + k, weight C(N, k)
                int sl = slot0 + k;
                sl = sl >= N ? sl - N : sl;
                const uint32_t q = ring[sl * C::PAIRS + i];
                lo += binom<N>(k) * (int)(q & 0xffffu);
                hi += binom<N>(k) * (int)(q >> 16);
            }
            *reinterpret_cast<int2 *>(Z + r * SC + c) = make_int2(lo, hi);
        }
        ring[slot0 * C::PAIRS + i] = g;
        c += C_STEP;
        r += R_STEP;
        if (c >= SC) {
            c -= SC;
            ++r;
        }
    }
}

// pass B (K3): G over rows 0..X+1, columns 0..X+3 from Z (Z column j is image column
// x0-4+j, Z row i image row y0-2+i); work items of SEG_B rows x 4 columns
template <int X>
__device__ __forceinline__ void pass_b(const int32_t *Z, int32_t *G)
{
    using C = BoxCfg<X>;
    constexpr int SR = C::SR, SC = C::SC, GW = C::GW, SEG = C::SEG_B;
    constexpr int GCOLS = GW / 4, SEGS = (X + 2 + SEG - 1) / SEG;
    for (int it = threadIdx.x; it < GCOLS * SEGS; it += C::THREADS) {
        const int g = 4 * (it % GCOLS), r0 = (it / GCOLS) * SEG;
        int hm2[4] = {0, 0, 0, 0}, hm1[4] = {0, 0, 0, 0};
#pragma unroll(C::UNROLL_B)
        for (int q = 0; q < SEG + 2; ++q) {
            const int i = min(r0 + q, SR - 1);  // rows past the plane only feed unstored G rows
            const int2 z01 = *reinterpret_cast<const int2 *>(Z + i * SC + g + 2);
            const int4 z25 = *reinterpret_cast<const int4 *>(Z + i * SC + g + 4);
            const int z[6] = {z01.x, z01.y, z25.x, z25.y, z25.z, z25.w};
            int h[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) h[c] = z[c] + 2 * z[c + 1] + z[c + 2];
            if (q >= 2 && r0 + q - 2 < X + 2) {
                int4 o;
                o.x = hm2[0] + 2 * hm1[0] + h[0];
                o.y = hm2[1] + 2 * hm1[1] + h[1];
                o.z = hm2[2] + 2 * hm1[2] + h[2];
                o.w = hm2[3] + 2 * hm1[3] + h[3];
                *reinterpret_cast<int4 *>(G + (r0 + q - 2) * GW + g) = o;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                hm2[c] = hm1[c];
                hm1[c] = h[c];
            }
        }
    }
}

// pass C (K4, K5): Sobel magnitude, threshold, mask and count of frame f over X * X
// outputs; work items of SEG_C rows x 4 columns. K4 clamps its own input: G rows and
// columns outside the frame read the nearest G inside it.
template <int N, int X>
__device__ __forceinline__ void pass_c(const StParams &p, const BoxPos &b, const int32_t *G, int f)
{
    using C = BoxCfg<X>;
    constexpr int GW = C::GW, SEG = C::SEG_C;
    constexpr int OCOLS = X / 4, SEGS = (X + SEG - 1) / SEG;
    const int thr = 261120 << N;
    int count = 0;
    uint8_t *mframe = p.mask + (int64_t)f * p.mask_fstride;
    for (int it = threadIdx.x; it < OCOLS * SEGS; it += C::THREADS) {
        const int o = 4 * (it % OCOLS), r0 = (it / OCOLS) * SEG;
        const bool clamp_cols = o < b.g_lo || o + 5 > b.g_hi;
        int dxm2[4] = {0, 0, 0, 0}, dxm1[4] = {0, 0, 0, 0}, sxm2[4] = {0, 0, 0, 0}, sxm1[4] = {0, 0, 0, 0};
#pragma unroll(C::UNROLL_C)
        for (int q = 0; q < SEG + 2; ++q) {  // G row r0+q; output row r0+q-2 centred on r0+q-1
            const int32_t *grow = G + min(max(r0 + q, b.gr_lo), b.gr_hi) * GW;
            int v[6];
            if (!clamp_cols) {
                const int4 a = *reinterpret_cast<const int4 *>(grow + o);
                const int2 c2 = *reinterpret_cast<const int2 *>(grow + o + 4);
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = c2.x; v[5] = c2.y;
            } else {
#pragma unroll
                for (int j = 0; j < 6; ++j) v[j] = grow[min(max(o + j, b.g_lo), b.g_hi)];
            }
            int dx[4], sx[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                dx[c] = v[c + 2] - v[c];
                sx[c] = v[c] + 2 * v[c + 1] + v[c + 2];
            }
            const int r = r0 + q - 2;
            if (q >= 2 && r < X) {
                uint32_t bits = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int gx = dxm2[c] + 2 * dxm1[c] + dx[c];
                    const int gy = sx[c] - sxm2[c];
                    bits |= (uint32_t)(abs(gx) + abs(gy) > thr) << (8 * c);
                }
                const int yy = b.y0 + r, xx = b.x0 + o;
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
    if ((threadIdx.x & 31) == 0 && count) atomicAdd(p.counts + f, count);
}

// Two barriers per frame: phase A runs pass C of the previous output frame, then waits
// for the staged frame and converts it; phase B issues the next frame's copy and runs
// pass B. The copy of frame pl+1 thus overlaps pass B of pl and pass C of pl.
template <int N, int X>
__global__ void __launch_bounds__(BoxCfg<X>::THREADS, 2) st_box_kernel(const __grid_constant__ StParams p)
{
    using C = BoxCfg<X>;
    extern __shared__ __align__(128) unsigned char st_smem[];
    // 128-byte aligned start (TMA destination), offset within the shared window so that
    // every pointer below stays a shared-memory pointer
    unsigned char *base = st_smem + ((128u - (smem_addr(st_smem) & 127u)) & 127u);
    const uint32_t *stage = reinterpret_cast<const uint32_t *>(base);
    int32_t *Z = reinterpret_cast<int32_t *>(base + C::OFF_Z);
    int32_t *G = reinterpret_cast<int32_t *>(base + C::OFF_G);
    uint32_t *ring = reinterpret_cast<uint32_t *>(base + C::OFF_RING);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + C::template off_bar<N>());

    const int nb_xy = p.boxes_x * p.boxes_y;
    const int bt = blockIdx.x / nb_xy, bxy = blockIdx.x - bt * nb_xy;
    const int by = bxy / p.boxes_x, bx = bxy - by * p.boxes_x;
    BoxPos b;
    b.x0 = bx * X;
    b.y0 = by * X;
    const int t0 = bt * p.t;
    const int t_end = min(t0 + p.t, p.T);
    const int n_planes = t_end - (t0 - N);  // the N frames before the box, then its own
    b.inner = b.x0 - 4 >= 0 && b.x0 + X + 4 <= p.W && b.y0 - 2 >= 0 && b.y0 + X + 2 <= p.H;
    b.gr_lo = b.y0 == 0 ? 1 : 0;
    b.gr_hi = min(X + 1, p.H - b.y0);
    b.g_lo = b.x0 == 0 ? 1 : 0;
    b.g_hi = min(X + 1, p.W - b.x0);

    if (threadIdx.x == 0) {
        bar_init(bar);
        bar_expect(bar, C::STAGE_BYTES);
        tma_frame(base, &p.tmap, b.x0 - 4, b.y0 - 2, max(t0 - N, 0), bar);
    }
    __syncthreads();

    // The pixel pairs a thread converts are the same in every frame (pair i by thread
    // i % THREADS), so the gray values of their N previous frames -- the temporal halo --
    // sit in a ring that only that thread touches: pair i of plane q in ring[(q % N) *
    // PAIRS + i]. No barrier guards it.
    for (int pl = 0; pl < n_planes; ++pl) {
        if (pl > N) pass_c<N, X>(p, b, G, t0 - N + pl - 1);
        const bool ok = bar_wait(bar, (unsigned)(pl & 1), p.wait_polls);
        if (ok) convert_frame<N, X>(p, b, stage, ring, Z, pl);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(p.err, ST_DEVERR_TIMEOUT);
                bar_wait(bar, (unsigned)(pl & 1));  // the copy in flight, once more (bounded)
            }
            return;
        }
        if (threadIdx.x == 0 && pl + 1 < n_planes) {
            bar_expect(bar, C::STAGE_BYTES);
            tma_frame(base, &p.tmap, b.x0 - 4, b.y0 - 2, max(t0 - N + pl + 1, 0), bar);
        }
        if (pl >= N) pass_b<X>(Z, G);
        __syncthreads();
    }
    if (n_planes > N) pass_c<N, X>(p, b, G, t_end - 1);
}

// the supported box sides and the kernel of (n, x); nullptr if not supported
using BoxKernel = void (*)(StParams);
template <int N> BoxKernel box_kernel_n(int x)
{
    switch (x) {
    case 8: return st_box_kernel<N, 8>;
    case 16: return st_box_kernel<N, 16>;
    case 32: return st_box_kernel<N, 32>;
    case 48: return st_box_kernel<N, 48>;
    case 64: return st_box_kernel<N, 64>;
    case 96: return st_box_kernel<N, 96>;
    default: return nullptr;
    }
}
BoxKernel box_kernel(int n, int x)
{
    return n == 1 ? box_kernel_n<1>(x) : n == 2 ? box_kernel_n<2>(x) : n == 4 ? box_kernel_n<4>(x) : nullptr;
}
int box_threads(int x)
{
    switch (x) {
    case 8: return BoxCfg<8>::THREADS;
    case 16: return BoxCfg<16>::THREADS;
    case 32: return BoxCfg<32>::THREADS;
    case 48: return BoxCfg<48>::THREADS;
    case 64: return BoxCfg<64>::THREADS;
    case 96: return BoxCfg<96>::THREADS;
    default: return 0;
    }
}
template <int N> int box_smem_n(int x)
{
    switch (x) {
    case 8: return BoxCfg<8>::smem<N>();
    case 16: return BoxCfg<16>::smem<N>();
    case 32: return BoxCfg<32>::smem<N>();
    case 48: return BoxCfg<48>::smem<N>();
    case 64: return BoxCfg<64>::smem<N>();
    case 96: return BoxCfg<96>::smem<N>();
    default: return 0;
    }
}
int box_smem(int n, int x) { return n == 1 ? box_smem_n<1>(x) : n == 2 ? box_smem_n<2>(x) : box_smem_n<4>(x); }

bool valid_n(int n) { return n == 1 || n == 2 || n == 4; }

}  // namespace

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
    if (!bytes || !kf::box_kernel(n, x)) return KF_EINVAL;
    *bytes = (size_t)kf::box_smem(n, x);
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
    if (!ctx || !video || t < 1) return KF_EINVAL;
    const kf::BoxKernel kern = kf::box_kernel(n, x);
    if (!kern) return KF_EINVAL;
    const int64_t W = video->W, H = video->H, T = video->T;
    if (W < 1 || H < 1 || T < 0 || W > 0x7fffffff || H > 0x7fffffff || T > 0x7fffffff) return KF_EINVAL;
    if (T == 0) return KF_OK;
    if (!video->rgba || !mask || !counts || (uintptr_t)video->rgba % 16 || (uintptr_t)mask % 16) return KF_EINVAL;
    if (video->pitch < W || video->pitch % 4 || mask_pitch < W || mask_pitch % 4) return KF_EINVAL;
    const int smem = kf::box_smem(n, x);
    if (smem > kf::ST_MAX_SMEM) return KF_EINVAL;
    const int64_t bxn = (W + x - 1) / x, byn = (H + x - 1) / x, btn = (T + t - 1) / t;
    if (bxn * byn * btn > 0x7fffffff) return KF_EINVAL;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
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
    p.wait_polls = ctx->wait_polls;
    p.W = (int)W;
    p.H = (int)H;
    p.T = (int)T;
    p.t = t;
    p.boxes_x = (int)bxn;
    p.boxes_y = (int)byn;
    const int threads = kf::box_threads(x);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)T, s);
    if (e != cudaSuccess) return st_fail(ctx, e);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return st_fail(ctx, e);
    kern<<<(unsigned)(bxn * byn * btn), threads, smem, s>>>(p);
    e = cudaGetLastError();
    return e == cudaSuccess ? KF_OK : st_fail(ctx, e);
}

kf_status kf_st_plan_eq6(double beta, int n, int *x, int *t)
{
    if (!(beta >= 1) || !kf::valid_n(n) || !x || !t) return KF_EINVAL;
    double xe = 0, te = 0;
    kf_st_box_eq6(beta, n, &xe, &te);
    static const int sides[] = {8, 16, 32, 48, 64, 96};
    int best = 8;
    double best_r = INFINITY;
    for (int sd : sides) {  // nearest supported side by ratio
        const double r = sd > xe ? sd / xe : xe / sd;
        if (r < best_r) {
            best_r = r;
            best = sd;
        }
    }
    *x = best;
    const double tt = beta / ((double)best * best);
    *t = tt < 1.0 ? 1 : (int)llround(tt);
    return KF_OK;
}

kf_status kf_st_tune(kf_ctx *ctx, const kf_pc_video *video, uint8_t *mask, int64_t mask_pitch, int32_t *counts, int n,
                     const int *boxes, int count, int reps, void *stream, int *best_x, int *best_t, float *best_ms)
{
    if (!ctx || !video || !boxes || count < 1 || reps < 1 || !best_x || !best_t) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    for (int i = 0; i < count; ++i)
        if (!kf::box_kernel(n, boxes[2 * i]) || boxes[2 * i + 1] < 1) return KF_EINVAL;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return st_fail(ctx, e);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return KF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KF_ECUDA;
    }
    int bx = 0, bt = 0;
    float best = INFINITY;
    kf_status st = KF_OK;
    for (int i = 0; i < count && st == KF_OK; ++i) {
        const int x = boxes[2 * i], t = boxes[2 * i + 1];
        st = kf_st_run(ctx, video, mask, mask_pitch, counts, n, x, t, stream);  // warm-up
        if (st != KF_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == KF_OK; ++r) st = kf_st_run(ctx, video, mask, mask_pitch, counts, n, x, t, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = KF_ECUDA;
        float ms = 0;
        if (st == KF_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / reps < best) {
            best = ms / reps;
            bx = x;
            bt = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KF_OK) return st;
    *best_x = bx;
    *best_t = bt;
    if (best_ms) *best_ms = best;
    return KF_OK;
}

}  // extern "C"
