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
//   2. lk_kernel: per selected point of frame t >= 1 (one half-warp each), one Lucas-Kanade step against
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

// the video of global frame g: the last v with frame_begin <= g
__device__ __forceinline__ const TrackVideo &video_of(const TrackVideo &one, const TrackVideo *vids, int n, int64_t g)
{
    if (!vids) return one;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (vids[mid].frame_begin <= g) lo = mid; else hi = mid - 1;
    }
    return vids[lo];
}

__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const TrackVideo one, const TrackVideo *vids, int n_videos,
                                                             int K)
{
    const TrackVideo &vd = video_of(one, vids, n_videos, blockIdx.x);
    const int frame = (int)(blockIdx.x - vd.frame_begin);
    const int tid = threadIdx.x;
    const int cap = vd.cand_cap;
    int32_t *n_points = vd.n_points, *idx_out = vd.idx;
    __shared__ unsigned hist[256];
    __shared__ unsigned long long sel[MAX_K];
    __shared__ unsigned nsel;
    __shared__ int digit_s, rank_s;
    if (frame == 0) {  // no previous frame: nothing to track
        if (tid == 0) n_points[0] = 0;
        return;
    }
    const unsigned long long *keys = vd.cand + (int64_t)frame * cap;
    const int n = min(vd.cand_count[frame], cap);
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

constexpr unsigned FULLM = 0xffffffffu;
constexpr int LK_WARPS = 4;  // warps per block; each half-warp (16 lanes) takes one point

// One half-warp per point. The clamped rows and columns within 4 of the point form a grid
// of nr x nc (<= 9 x 9) positions that holds every smoothed value the 7x7 window and its
// Sobel neighbours read. Lane j < nq of the half computes the horizontal Gaussian of frame
// row q0 + j on the grid columns; lane i < nr gathers its five vertical taps by shuffles
// and holds smoothed grid row r0 + i; lane d < 7 accumulates window row d - 3. All values
// up to the Sobel output are integers below 2^24, exact in FP32 and equal to the chain's.
__global__ void __launch_bounds__(32 * LK_WARPS) lk_kernel(const TrackVideo one, const TrackVideo *vids, int n_videos,
                                                           int64_t total_frames, int K)
{
    const int lane = threadIdx.x & 15;  // lane within the half-warp
    const int64_t gid = ((int64_t)blockIdx.x * LK_WARPS + (threadIdx.x >> 5)) * 2 + ((threadIdx.x >> 4) & 1);
    const int64_t gframe = gid / K;
    const int i = (int)(gid % K);
    const TrackVideo &vd = video_of(one, vids, n_videos, min(gframe, total_frames - 1));
    const int frame_g = (int)(gframe - vd.frame_begin);
    const int W = vd.W, H = vd.H;
    const int64_t pitch = vd.pitch;
    const bool valid = gframe < total_frames && frame_g > 0 && i < vd.n_points[frame_g];
    if (!__any_sync(FULLM, valid)) return;  // warp-uniform
    // an idle half works on a stand-in point (row 0, column 0 of its video's frame 0,
    // against itself) and stores nothing
    const int frame = valid ? frame_g : 0;
    const int p = valid ? vd.idx[(int64_t)frame_g * K + i] : 0;
    const int py = p / W, px = p % W;
    const int r0 = max(py - 4, 0), nr = min(py + 4, H - 1) - r0 + 1;
    const int c0 = max(px - 4, 0), nc = min(px + 4, W - 1) - c0 + 1;
    const int q0 = max(r0 - 2, 0), nq = min(r0 + nr - 1 + 2, H - 1) - q0 + 1;
    const int64_t fstride = (int64_t)H * pitch;
    const uint8_t *fc = vd.frames + (int64_t)frame * fstride, *fp = frame > 0 ? fc - fstride : fc;

    // horizontal pass: lane j holds g1 of row q0 + j (both frames) on the grid columns;
    // the lane loads the 13 clamped bytes of its row once per frame
    float h_c[9], h_p[9];
    {
        const int y = q0 + min(lane, nq - 1);
        const uint8_t *rc = fc + (int64_t)y * pitch, *rp = fp + (int64_t)y * pitch;
        float bc[13], bp[13];
#pragma unroll
        for (int j = 0; j < 13; ++j) {  // byte j: column c0 - 2 + j, clamped
            const int x = clampi(c0 - 2 + j, 0, W - 1);
            bc[j] = (float)rc[x];
            bp[j] = (float)rp[x];
        }
        const bool inner = (c0 >= 2) && (c0 + 10 <= W - 1);  // no clamping inside the 13 bytes
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            if (inner) {
                float t = bc[j] + bc[j + 4];
                t = fmaf(4.0f, bc[j + 1] + bc[j + 3], t);
                h_c[j] = fmaf(6.0f, bc[j + 2], t);
                float u = bp[j] + bp[j + 4];
                u = fmaf(4.0f, bp[j + 1] + bp[j + 3], u);
                h_p[j] = fmaf(6.0f, bp[j + 2], u);
            } else {  // grid column x = c0 + j (clamped to the grid) and its clamped taps
                const int x = c0 + min(j, nc - 1);
                float t = (float)rc[clampi(x - 2, 0, W - 1)] + (float)rc[clampi(x + 2, 0, W - 1)];
                t = fmaf(4.0f, (float)rc[clampi(x - 1, 0, W - 1)] + (float)rc[clampi(x + 1, 0, W - 1)], t);
                h_c[j] = fmaf(6.0f, (float)rc[x], t);
                float u = (float)rp[clampi(x - 2, 0, W - 1)] + (float)rp[clampi(x + 2, 0, W - 1)];
                u = fmaf(4.0f, (float)rp[clampi(x - 1, 0, W - 1)] + (float)rp[clampi(x + 1, 0, W - 1)], u);
                h_p[j] = fmaf(6.0f, (float)rp[x], u);
            }
        }
    }
    // vertical pass: lane i holds smoothed row r0 + i
    float g_c[9], g_p[9];
    {
        const int y = r0 + min(lane, nr - 1);
        int src[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) src[k] = clampi(y + k - 2, 0, H - 1) - q0;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            float a[5], b[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                a[k] = __shfl_sync(FULLM, h_c[j], src[k], 16);
                b[k] = __shfl_sync(FULLM, h_p[j], src[k], 16);
            }
            g_c[j] = (a[0] + a[4]) + 4.0f * (a[1] + a[3]) + 6.0f * a[2];
            g_p[j] = (b[0] + b[4]) + 4.0f * (b[1] + b[3]) + 6.0f * b[2];
        }
    }
    // window row d = lane - 3 (lanes 0..6): Sobel rows ym, y0, yp of the clamped window row
    const int dy = min(lane, 6) - 3;
    const int qy = clampi(py + dy, 0, H - 1);
    const int lm = clampi(qy - 1, 0, H - 1) - r0, l0 = qy - r0, lp = clampi(qy + 1, 0, H - 1) - r0;
    float gm[9], gz[9], gq[9], gpz[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        gm[j] = __shfl_sync(FULLM, g_c[j], lm, 16);
        gz[j] = __shfl_sync(FULLM, g_c[j], l0, 16);
        gq[j] = __shfl_sync(FULLM, g_c[j], lp, 16);
        gpz[j] = __shfl_sync(FULLM, g_p[j], l0, 16);
    }
    float a00 = 0, a01 = 0, a11 = 0, b0 = 0, b1 = 0;
    auto accumulate = [&](float vm_m, float vm_0, float vm_q, float vz_m, float vz_0, float vz_q, float vq_m, float vq_0,
                          float vq_q, float vp_0) {
        const float ix = (vm_q - vm_m) + 2.0f * (vz_q - vz_m) + (vq_q - vq_m);
        const float iy = (vq_m - vm_m) + 2.0f * (vq_0 - vm_0) + (vq_q - vm_q);
        const float it = vz_0 - vp_0;
        a00 = fmaf(ix, ix, a00);
        a01 = fmaf(ix, iy, a01);
        a11 = fmaf(iy, iy, a11);
        b0 = fmaf(ix, it, b0);
        b1 = fmaf(iy, it, b1);
    };
    if (lane < 7) {
        if (px >= 4 && px <= W - 5) {  // no column clamping: grid column of dx is dx + 4
#pragma unroll
            for (int dx = -3; dx <= 3; ++dx) {
                const int m = dx + 3, z = dx + 4, q = dx + 5;
                accumulate(gm[m], gm[z], gm[q], gz[m], gz[z], gz[q], gq[m], gq[z], gq[q], gpz[z]);
            }
        } else {
#pragma unroll
            for (int dx = -3; dx <= 3; ++dx) {
                const int qx = clampi(px + dx, 0, W - 1);
                const int xm = clampi(qx - 1, 0, W - 1) - c0, x0 = qx - c0, xq = clampi(qx + 1, 0, W - 1) - c0;
                // columns are runtime indices into 9-element rows: select without local memory
                float vm_m = 0, vm_q = 0, vz_m = 0, vz_0 = 0, vz_q = 0, vq_m = 0, vq_0 = 0, vq_q = 0, vm_0 = 0, vp_0 = 0;
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    vm_m = j == xm ? gm[j] : vm_m; vm_0 = j == x0 ? gm[j] : vm_0; vm_q = j == xq ? gm[j] : vm_q;
                    vz_m = j == xm ? gz[j] : vz_m; vz_0 = j == x0 ? gz[j] : vz_0; vz_q = j == xq ? gz[j] : vz_q;
                    vq_m = j == xm ? gq[j] : vq_m; vq_0 = j == x0 ? gq[j] : vq_0; vq_q = j == xq ? gq[j] : vq_q;
                    vp_0 = j == x0 ? gpz[j] : vp_0;
                }
                accumulate(vm_m, vm_0, vm_q, vz_m, vz_0, vz_q, vq_m, vq_0, vq_q, vp_0);
            }
        }
    }
    // sum the 7 window rows (fixed order: lanes 0..6 by a tree within the warp)
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
        a00 += __shfl_down_sync(FULLM, a00, off, 16);
        a01 += __shfl_down_sync(FULLM, a01, off, 16);
        a11 += __shfl_down_sync(FULLM, a11, off, 16);
        b0 += __shfl_down_sync(FULLM, b0, off, 16);
        b1 += __shfl_down_sync(FULLM, b1, off, 16);
    }
    if (lane != 0 || !valid) return;
    // scaled units: gx = ix / (8 s), gt = it / s with s = 65280, so -A^-1 b = -8 A'^-1 b'
    const int64_t o = (int64_t)frame_g * K + i;
    const double A00 = a00, A01 = a01, A11 = a11, B0 = b0, B1 = b1;
    const double det = A00 * A11 - A01 * A01;
    const double tr = A00 + A11;
    if (fabs(det) <= 1e-12 * tr * tr) {
        vd.u[o] = 0.0f;
        vd.v[o] = 0.0f;
        vd.status[o] = 1;
    } else {
        vd.u[o] = (float)(-8.0 * (A11 * B0 - A01 * B1) / det);
        vd.v[o] = (float)(-8.0 * (A00 * B1 - A01 * B0) / det);
        vd.status[o] = 0;
    }
}

}  // namespace

int launch_select(const TrackVideo &one, const TrackVideo *vids, int n, int64_t total_frames, int K, void *stream)
{
    if (K < 1 || K > MAX_K || total_frames > 0x7fffffff) return (int)cudaErrorInvalidValue;
    if (total_frames == 0) return 0;
    select_kernel<<<(unsigned)total_frames, SEL_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(one, vids, n, K);
    return (int)cudaGetLastError();
}

int launch_lk(const TrackVideo &one, const TrackVideo *vids, int n, int64_t total_frames, int K, void *stream)
{
    const int64_t slots = total_frames * K;
    if (slots == 0) return 0;
    const unsigned blocks = (unsigned)((slots + 2 * LK_WARPS - 1) / (2 * LK_WARPS));
    lk_kernel<<<blocks, 32 * LK_WARPS, 0, static_cast<cudaStream_t>(stream)>>>(one, vids, n, total_frames, K);
    return (int)cudaGetLastError();
}

}  // namespace kf
