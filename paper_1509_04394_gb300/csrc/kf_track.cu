// kf_track.cu -- the temporal stages: feature selection and one Lucas-Kanade step.
//
// Tracking reads whole-frame results of the corner chain (the K strongest corners of a
// frame), so it depends on every block of the previous kernel: a kernel-to-kernel
// dependency (Sec. V-A c) that ends the chain's fusable set, like the Kalman step of
// Table IV. It therefore runs as separate kernels after the fused chain:
//   1. select_kernel: per frame, the K largest corner keys among the candidates the
//      fused chain appended (key = R bits << 32 | ~raster index, so larger keys are
//      stronger corners and, at equal R, lower raster indices); an exact MSB-first radix
//      select (8 passes of 8 bits) finds the K-th largest key, a bitonic sort orders the
//      winners;
//   2. lk_kernel: per selected point of frame t >= 1, one Lucas-Kanade step against
//      frame t-1 over a 7x7 window: A = sum [gx^2, gx gy; gx gy, gy^2],
//      b = sum [gx gt, gy gt], (u, v) = -A^-1 b, gx, gy = Sobel of the smoothed frame t
//      over 8, gt = difference of the smoothed frames. The smoothed patches are recomputed
//      from the u8 frames in the chain's integer-scaled units (exact in FP32, identical to
//      the chain's maps); the window sums are FP32; the determinant, the singularity
//      test |det| <= 1e-12 (A00 + A11)^2 and the 2x2 solve are FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kf_params.h"

namespace kf {
namespace {

constexpr int SEL_THREADS = 256;
constexpr int MAX_K = 1024;

__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const unsigned long long *cand, const int *cand_count,
                                                             int cap, int K, int32_t *n_points, int32_t *idx_out)
{
    const int frame = blockIdx.x;
    const int tid = threadIdx.x;
    __shared__ unsigned hist[256];
    __shared__ unsigned long long sel[MAX_K];
    __shared__ unsigned nsel;
    __shared__ int digit_s, rank_s;
    if (frame == 0) {  // no previous frame: nothing to track
        if (tid == 0) n_points[0] = 0;
        return;
    }
    const unsigned long long *keys = cand + (int64_t)frame * cap;
    const int n = min(cand_count[frame], cap);
    const int kk = min(n, K);
    unsigned long long kth = 0;  // every key >= kth is selected
    if (n > K) {
        unsigned long long prefix = 0, pmask = 0;
        int rank = K;  // rank of the wanted key among those matching the prefix (1 = largest)
        for (int pass = 0; pass < 8; ++pass) {
            const int shift = 56 - 8 * pass;
            for (int d = tid; d < 256; d += SEL_THREADS) hist[d] = 0;
            __syncthreads();
            for (int i = tid; i < n; i += SEL_THREADS) {
                const unsigned long long k = keys[i];
                if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255], 1u);
            }
            __syncthreads();
            if (tid == 0) {
                int cum = 0, d = 255;
                for (; d > 0; --d) {
                    if (cum + (int)hist[d] >= rank) break;
                    cum += hist[d];
                }
                digit_s = d;
                rank_s = rank - cum;
            }
            __syncthreads();
            prefix |= (unsigned long long)digit_s << shift;
            pmask |= 0xffull << shift;
            rank = rank_s;
            __syncthreads();
        }
        kth = prefix;  // keys are distinct, so exactly K keys are >= kth
    }
    if (tid == 0) nsel = 0;
    __syncthreads();
    for (int i = tid; i < n; i += SEL_THREADS) {
        const unsigned long long k = keys[i];
        if (k >= kth) {
            const unsigned pos = atomicAdd(&nsel, 1u);
            if (pos < (unsigned)MAX_K) sel[pos] = k;
        }
    }
    __syncthreads();
    int P = 1;
    while (P < kk) P <<= 1;
    for (int i = kk + tid; i < P; i += SEL_THREADS) sel[i] = 0;  // padding sorts last
    __syncthreads();
    // bitonic sort, descending
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < P; i += SEL_THREADS) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool desc = (i & size) == 0;
                    const unsigned long long a = sel[i], b = sel[j];
                    if ((a < b) == desc) {
                        sel[i] = b;
                        sel[j] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = tid; i < kk; i += SEL_THREADS) idx_out[(int64_t)frame * K + i] = (int32_t)(0xffffffffu - (unsigned)sel[i]);
    if (tid == 0) n_points[frame] = kk;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// smoothed frame g (scaled by 65280, exact) on the grid rows [r0, r0+nr) x cols [c0, c0+nc)
__device__ void smooth_grid(const uint8_t *f, int64_t pitch, int W, int H, int r0, int nr, int c0, int nc, float (&g)[9][9])
{
    // horizontal pass on the rows the vertical pass reads (clamped), the chain's order
    const int q0 = max(r0 - 2, 0), q1 = min(r0 + nr - 1 + 2, H - 1);
    float g1[13][9];
    for (int y = q0; y <= q1; ++y) {
        const uint8_t *row = f + (int64_t)y * pitch;
        for (int j = 0; j < nc; ++j) {
            const int x = c0 + j;
            const float a = row[clampi(x - 2, 0, W - 1)], b = row[clampi(x - 1, 0, W - 1)], c = row[x],
                        d = row[clampi(x + 1, 0, W - 1)], e = row[clampi(x + 2, 0, W - 1)];
            float t = a + e;
            t = fmaf(4.0f, b + d, t);
            g1[y - q0][j] = fmaf(6.0f, c, t);
        }
    }
    for (int i = 0; i < nr; ++i) {
        const int y = r0 + i;
        for (int j = 0; j < nc; ++j) {
            const float a = g1[clampi(y - 2, 0, H - 1) - q0][j], b = g1[clampi(y - 1, 0, H - 1) - q0][j], c = g1[y - q0][j],
                        d = g1[clampi(y + 1, 0, H - 1) - q0][j], e = g1[clampi(y + 2, 0, H - 1) - q0][j];
            g[i][j] = (a + e) + 4.0f * (b + d) + 6.0f * c;  // integers < 2^24: exact in any order
        }
    }
}

__global__ void __launch_bounds__(128) lk_kernel(const uint8_t *frames, int64_t pitch, int W, int H, int T, int K,
                                                 const int32_t *n_points, const int32_t *idx, float *u_out, float *v_out,
                                                 int32_t *status)
{
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)T * K) return;
    const int frame = (int)(gid / K), i = (int)(gid % K);
    if (frame == 0 || i >= n_points[frame]) return;
    const int p = idx[gid];
    const int py = p / W, px = p % W;
    // grid of the clamped rows/columns within 4 of the point: holds every g the 7x7
    // window and its Sobel neighbours read
    const int r0 = max(py - 4, 0), nr = min(py + 4, H - 1) - r0 + 1;
    const int c0 = max(px - 4, 0), nc = min(px + 4, W - 1) - c0 + 1;
    float gt[9][9], gp[9][9];
    const int64_t fstride = (int64_t)H * pitch;
    smooth_grid(frames + (int64_t)frame * fstride, pitch, W, H, r0, nr, c0, nc, gt);
    smooth_grid(frames + (int64_t)(frame - 1) * fstride, pitch, W, H, r0, nr, c0, nc, gp);
    float a00 = 0, a01 = 0, a11 = 0, b0 = 0, b1 = 0;
    for (int dy = -3; dy <= 3; ++dy) {
        const int qy = clampi(py + dy, 0, H - 1);
        const int ym = clampi(qy - 1, 0, H - 1) - r0, y0 = qy - r0, yp = clampi(qy + 1, 0, H - 1) - r0;
        for (int dx = -3; dx <= 3; ++dx) {
            const int qx = clampi(px + dx, 0, W - 1);
            const int xm = clampi(qx - 1, 0, W - 1) - c0, x0 = qx - c0, xq = clampi(qx + 1, 0, W - 1) - c0;
            const float ix = (gt[ym][xq] - gt[ym][xm]) + 2.0f * (gt[y0][xq] - gt[y0][xm]) + (gt[yp][xq] - gt[yp][xm]);
            const float iy = (gt[yp][xm] - gt[ym][xm]) + 2.0f * (gt[yp][x0] - gt[ym][x0]) + (gt[yp][xq] - gt[ym][xq]);
            const float it = gt[y0][x0] - gp[y0][x0];
            a00 = fmaf(ix, ix, a00);
            a01 = fmaf(ix, iy, a01);
            a11 = fmaf(iy, iy, a11);
            b0 = fmaf(ix, it, b0);
            b1 = fmaf(iy, it, b1);
        }
    }
    // scaled units: gx = ix / (8 s), gt = it / s with s = 65280, so -A^-1 b = -8 A'^-1 b'
    const double A00 = a00, A01 = a01, A11 = a11, B0 = b0, B1 = b1;
    const double det = A00 * A11 - A01 * A01;
    const double tr = A00 + A11;
    if (fabs(det) <= 1e-12 * tr * tr) {
        u_out[gid] = 0.0f;
        v_out[gid] = 0.0f;
        status[gid] = 1;
    } else {
        u_out[gid] = (float)(-8.0 * (A11 * B0 - A01 * B1) / det);
        v_out[gid] = (float)(-8.0 * (A00 * B1 - A01 * B0) / det);
        status[gid] = 0;
    }
}

}  // namespace

int launch_select(const unsigned long long *cand, const int *cand_count, int cap, int K, int T, int32_t *n_points,
                  int32_t *idx, void *stream)
{
    if (K < 1 || K > MAX_K) return (int)cudaErrorInvalidValue;
    select_kernel<<<T, SEL_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(cand, cand_count, cap, K, n_points, idx);
    return (int)cudaGetLastError();
}

int launch_lk(const uint8_t *frames, int64_t pitch, int W, int H, int T, int K, const int32_t *n_points,
              const int32_t *idx, float *u, float *v, int32_t *status, void *stream)
{
    const int64_t n = (int64_t)T * K;
    const unsigned blocks = (unsigned)((n + 127) / 128);
    lk_kernel<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(frames, pitch, W, H, T, K, n_points, idx, u, v, status);
    return (int)cudaGetLastError();
}

}  // namespace kf
