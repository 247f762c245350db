// kf_track.cu -- the temporal stages: feature selection and one Lucas-Kanade step.
//
// Tracking reads whole-frame results of the corner chain (the K strongest corners of a
// frame), so it depends on every block of the previous kernel: a kernel-to-kernel
// dependency (Sec. V-A c) that ends the chain's fusable set, like the Kalman step of
// Table IV. It therefore runs as separate kernels after the fused chain:
//   1. select_kernel: per frame, the K largest corner keys among the candidates the
//      fused chain appended (key = R bits << 32 | ~raster index, so larger keys are
//      stronger corners and, at equal R, lower raster indices). An exact MSB-first radix
//      select finds the K-th largest key: the pass that stages a frame's keys in shared
//      memory (when they fit) also histograms their top 9 bits (sign and exponent of R);
//      the exponent bucket holding the K-th key is gathered on chip, the keys of higher
//      buckets are winners, and 8-bit digits of the gathered bucket are histogrammed until
//      the bucket holding the K-th key is taken whole. The winners are then ordered by a
//      bitonic sort in shared memory;
//   2. lk_kernel: per selected point of frame t >= 1, one Lucas-Kanade step against
//      frame t-1 over a 7x7 window: A = sum [gx^2, gx gy; gx gy, gy^2],
//      b = sum [gx gt, gy gt], (u, v) = -A^-1 b, gx, gy = Sobel of the smoothed frame t
//      over 8, gt = difference of the smoothed frames. The smoothed patches are recomputed
//      from the u8 frames in the chain's integer-scaled units (exact, identical to the
//      chain's maps); the window sums are FP32; the determinant, the singularity test
//      |det| <= 1e-12 (A00 + A11)^2 and the 2x2 solve are FP64. A point whose 13x13 input
//      patch lies inside the frame is one thread's work (no clamping: packed 16-bit
//      integer Gaussian on word loads, FP32 Sobel and sums in registers); a point nearer
//      the border (clamped window) is done by half a warp on a clamped 9x9 grid.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kf_params.h"

namespace kf {
namespace {

constexpr unsigned FULLM = 0xffffffffu;
constexpr int SEL_THREADS = 512;
constexpr int SEL_SMEM_KEYS = 10240;  // a frame's keys are staged on chip up to this count (80 KiB)
constexpr int SEL_LIST = 2048;        // keys of the K-th key's exponent bucket, gathered on chip (16 KiB)
constexpr int SEL_DYN_BYTES = (SEL_SMEM_KEYS + SEL_LIST) * (int)sizeof(unsigned long long);
constexpr int MAX_K = 1024;
constexpr int MAX_DEVICES = 64;

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

// Warp 0: the bucket holding the rank-th largest key (1 = largest), from a histogram of
// NB buckets (lane l holds buckets NB/32 * l on): suffix sums over the lanes give each
// lane the count of keys in higher buckets. Writes the bucket, the rank within it and its
// count to sh[0..2].
template <int NB>
__device__ __forceinline__ void find_bucket(const unsigned *hist, int rank, int lane, int *sh)
{
    constexpr int PER = NB / 32;
    unsigned c[PER], s = 0;
#pragma unroll
    for (int b = 0; b < PER; ++b) {
        c[b] = hist[PER * lane + b];
        s += c[b];
    }
    unsigned incl = s;  // keys in this lane's buckets and above
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_down_sync(FULLM, incl, o);
        if (lane + o < 32) incl += y;
    }
    const unsigned above = incl - s;
    if (above < (unsigned)rank && (unsigned)rank <= incl) {
        unsigned cum = above, cnt = 0;
        int d = PER * lane;
#pragma unroll
        for (int b = PER - 1; b >= 0; --b) {
            if (cum + c[b] >= (unsigned)rank) {
                d = PER * lane + b;
                cnt = c[b];
                break;
            }
            cum += c[b];
        }
        sh[0] = d;
        sh[1] = rank - (int)cum;
        sh[2] = (int)cnt;
    }
}

// Block-wide append: the threads whose `take` holds put their key in list[] from *count on
// (one shared atomic per warp, lane order within the warp); every thread calls it.
__device__ __forceinline__ void append_key(bool take, unsigned long long k, unsigned long long *list, unsigned *count,
                                           int lane, unsigned cap)
{
    const unsigned b = __ballot_sync(FULLM, take);
    if (b) {  // warp-uniform
        unsigned pos = 0;
        if (lane == 0) pos = atomicAdd(count, (unsigned)__popc(b));
        pos = __shfl_sync(FULLM, pos, 0) + __popc(b & ((1u << lane) - 1u));
        if (take && pos < cap) list[pos] = k;
    }
}

// Block-wide MSB-first radix select: among the keys of keys[0..m) that equal `prefix` on
// the bits of `pmask` (every bit above `top`), the key kth such that exactly `rank` of them
// are >= kth. Each pass histograms the next 8-bit digit of the matching keys and keeps the
// bucket holding the rank-th largest; it ends when that bucket is taken whole (kth is then
// the bucket's smallest possible key) or every bit is fixed.
__device__ unsigned long long radix_kth(const unsigned long long *keys, int m, unsigned long long prefix,
                                        unsigned long long pmask, int top, int rank, unsigned *hist, int *sh)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        const int width = min(8, top + 1);
        const int shift = top + 1 - width;
        const unsigned dmask = (1u << width) - 1u;
        if (tid < 256) hist[tid] = 0;
        __syncthreads();
        for (int i = tid; i < m; i += SEL_THREADS) {
            const unsigned long long k = keys[i];
            if ((k & pmask) == prefix) atomicAdd(&hist[(unsigned)(k >> shift) & dmask], 1u);
        }
        __syncthreads();
        if (warp == 0) find_bucket<256>(hist, rank, lane, sh);
        __syncthreads();
        prefix |= (unsigned long long)sh[0] << shift;
        pmask |= (unsigned long long)dmask << shift;
        const bool whole = sh[1] == sh[2];
        rank = sh[1];
        top = shift - 1;
        // sh and hist are rewritten only after the next pass's first barrier
        if (whole || top < 0) return prefix;
    }
}

__global__ void __launch_bounds__(SEL_THREADS, 2) select_kernel(const TrackVideo one, const TrackVideo *vids, int n_videos,
                                                             int K)
{
    extern __shared__ unsigned long long skeys[];  // SEL_SMEM_KEYS staged keys, then SEL_LIST bucket keys
    unsigned long long *blist = skeys + SEL_SMEM_KEYS;
    __shared__ unsigned hist[512];
    __shared__ unsigned long long sel[MAX_K];
    __shared__ unsigned nsel, nlist;
    __shared__ int sh[3];
    const TrackVideo &vd = video_of(one, vids, n_videos, blockIdx.x);
    const int frame = (int)(blockIdx.x - vd.frame_begin + vd.first_frame);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cap = vd.cand_cap;
    int32_t *n_points = vd.n_points, *idx_out = vd.idx;
    if (frame == 0) {  // no previous frame: nothing to track
        if (tid == 0) n_points[0] = 0;
        return;
    }
    const unsigned long long *gkeys = vd.cand + (int64_t)frame * cap;
    const int n = min(vd.cand_count[frame], cap);
    const int kk = min(n, K);
    if (n > K) {
        const bool staged = n <= SEL_SMEM_KEYS;
        const unsigned long long *keys = staged ? skeys : gkeys;
        // pass 1: stage the keys (16-byte loads, 16 keys per thread in flight) and
        // histogram their top 9 bits, the sign and exponent of R
        for (int i = tid; i < 512; i += SEL_THREADS) hist[i] = 0;
        if (tid == 0) {
            nsel = 0;
            nlist = 0;
        }
        __syncthreads();
        const ulonglong2 *g2 = reinterpret_cast<const ulonglong2 *>(gkeys);
        const int n2 = n >> 1;
        for (int base = 0; base < n2; base += 8 * SEL_THREADS) {
            ulonglong2 k[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = base + u * SEL_THREADS + tid;
                k[u] = i < n2 ? g2[i] : make_ulonglong2(0ull, 0ull);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = base + u * SEL_THREADS + tid;
                const bool valid = i < n2;
                if (valid && staged) reinterpret_cast<ulonglong2 *>(skeys)[i] = k[u];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const unsigned d = (unsigned)((h ? k[u].y : k[u].x) >> 55);
                    if (valid) atomicAdd(&hist[d], 1u);
                }
            }
        }
        if ((n & 1) && tid == 0) {
            const unsigned long long k = gkeys[n - 1];
            if (staged) skeys[n - 1] = k;
            atomicAdd(&hist[(unsigned)(k >> 55)], 1u);
        }
        __syncthreads();
        if (warp == 0) find_bucket<512>(hist, K, lane, sh);
        __syncthreads();
        const unsigned dstar = (unsigned)sh[0];
        const int rank_in = sh[1], cnt = sh[2];
        const unsigned long long pfx = (unsigned long long)dstar << 55, pm = ~0ull << 55;
        unsigned long long kth = pfx;  // the bucket taken whole unless narrowed below
        if (cnt <= SEL_LIST) {
            // pass 2: keys of higher buckets are winners; the bucket's keys are gathered
            for (int base = 0; base < n; base += SEL_THREADS) {
                const int i = base + tid;
                const unsigned long long k = i < n ? keys[i] : 0ull;
                const unsigned d = (unsigned)(k >> 55);
                append_key(i < n && d > dstar, k, sel, &nsel, lane, MAX_K);
                append_key(i < n && d == dstar, k, blist, &nlist, lane, SEL_LIST);
            }
            __syncthreads();
            if (rank_in < cnt) kth = radix_kth(blist, cnt, pfx, pm, 54, rank_in, hist, sh);
            for (int base = 0; base < cnt; base += SEL_THREADS) {
                const int i = base + tid;
                const unsigned long long k = i < cnt ? blist[i] : 0ull;
                append_key(i < cnt && k >= kth, k, sel, &nsel, lane, MAX_K);
            }
        } else {  // a large bucket: the remaining passes over all keys
            if (rank_in < cnt) kth = radix_kth(keys, n, pfx, pm, 54, rank_in, hist, sh);
            for (int base = 0; base < n; base += SEL_THREADS) {
                const int i = base + tid;
                const unsigned long long k = i < n ? keys[i] : 0ull;
                append_key(i < n && k >= kth, k, sel, &nsel, lane, MAX_K);
            }
        }
    } else {
        for (int i = tid; i < n; i += SEL_THREADS) sel[i] = gkeys[i];  // every key is selected
    }
    // order: bitonic sort of the kk winners, descending (keys are distinct; the padding up
    // to a power of two is 0, below every key)
    int P = 1;
    while (P < kk) P <<= 1;
    __syncthreads();
    for (int i = kk + tid; i < P; i += SEL_THREADS) sel[i] = 0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < (P >> 1); i += SEL_THREADS) {
                const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                const unsigned long long a = sel[lo], b = sel[hi];
                const bool desc = (lo & size) == 0;  // every block descending at the last merge
                if (desc ? a < b : a > b) {
                    sel[lo] = b;
                    sel[hi] = a;
                }
            }
            __syncthreads();
        }
    }
    for (int t = tid; t < kk; t += SEL_THREADS) idx_out[(int64_t)frame * K + t] = (int32_t)(0xffffffffu - (unsigned)sel[t]);
    if (tid == 0) n_points[frame] = kk;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// The 2x2 solve of one point from its FP32 window sums (scaled units: gx = ix / (8 s),
// gt = it / s with s = 65280, so -A^-1 b = -8 A'^-1 b').
__device__ __forceinline__ void store_step(const TrackVideo &vd, int64_t o, float a00, float a01, float a11, float b0,
                                           float b1)
{
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

// ---- interior points: one thread, no clamping --------------------------------------------
//
// A packed word holds two 16-bit lanes, lo = the value at column c, hi = at c + 1. The
// binomial 5-tap sum of packed words is lane-wise exact: the horizontal sums of bytes are
// at most 16 * 255 and the vertical sums of those at most 65280 < 2^16, and every partial
// sum is below the total, so no lane carries into the next.
__device__ __forceinline__ unsigned binom5(unsigned a, unsigned b, unsigned c, unsigned d, unsigned e)
{
    return (a + e) + ((b + d) << 2) + c * 6u;
}
// lanes to FP32 (exact): the 16-bit value under the exponent of 2^23, minus 2^23
__device__ __forceinline__ float lo_f(unsigned x) { return __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7610)) - 8388608.0f; }
__device__ __forceinline__ float hi_f(unsigned x) { return __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7632)) - 8388608.0f; }

// Bytes b_0..b_12 of a row from column x0 on, as byte pairs P[j] = b_j | b_{j+1} << 16.
// `row` is the 4-byte aligned word holding column x0; sh = 8 (x0 mod 4).
__device__ __forceinline__ void row_pairs(const unsigned *row, int sh, unsigned P[13])
{
    const unsigned w0 = __ldg(row), w1 = __ldg(row + 1), w2 = __ldg(row + 2), w3 = __ldg(row + 3);
    const unsigned u0 = __funnelshift_r(w0, w1, sh), u1 = __funnelshift_r(w1, w2, sh), u2 = __funnelshift_r(w2, w3, sh),
                   u3 = w3 >> sh;
    P[0] = __byte_perm(u0, 0, 0x4140);
    P[2] = __byte_perm(u0, 0, 0x4342);
    P[4] = __byte_perm(u1, 0, 0x4140);
    P[6] = __byte_perm(u1, 0, 0x4342);
    P[8] = __byte_perm(u2, 0, 0x4140);
    P[10] = __byte_perm(u2, 0, 0x4342);
    P[12] = __byte_perm(u3, 0, 0x4140);
#pragma unroll
    for (int j = 1; j < 12; j += 2) P[j] = __funnelshift_r(P[j - 1], P[j + 1], 16);
}

constexpr int LK_THREADS = 128;  // one point per thread

// Window sums of an interior point (6 <= px <= W-7, 6 <= py <= H-7). Rows stream top to
// bottom: raw row s of frame t (y = py-6+s, s = 0..12) gives the packed horizontal
// Gaussian hc[s] on grid columns px-4..px+4; from s = 4 on, grid row s-4 (y = py-8+s)
// is complete and gives its Sobel partials D = g(x+1) - g(x-1), S = g(x-1) + 2 g(x) +
// g(x+1) on window columns px-3..px+3. Raw row s-2 of frame t-1 (y = py-7+s) gives hp;
// from s = 6 on, window row w = s-6 has its three grid rows and its t-1 row.
__device__ __forceinline__ void lk_sums_interior(const TrackVideo &vd, int frame, int px, int py, float acc[5])
{
    const int64_t pitch = vd.pitch;
    const int64_t fstride = (int64_t)vd.H * pitch;
    const int x0 = px - 6;
    const int sh = 8 * (x0 & 3);
    const uint8_t *cur = vd.frames + (int64_t)frame * fstride + (int64_t)(py - 6) * pitch + (x0 & ~3);
    const uint8_t *prv = cur - fstride + pitch;  // frame t-1, row py-5
    unsigned hc[13][5], hp[11][4];
    float D[9][7], S[9][7], Gm[9][7];
    float a00 = 0.f, a01 = 0.f, a11 = 0.f, b0 = 0.f, b1 = 0.f;
#pragma unroll
    for (int s = 0; s < 13; ++s) {
        {
            unsigned P[13];
            row_pairs(reinterpret_cast<const unsigned *>(cur + (int64_t)s * pitch), sh, P);
#pragma unroll
            for (int k = 0; k < 5; ++k) hc[s][k] = binom5(P[2 * k], P[2 * k + 1], P[2 * k + 2], P[2 * k + 3], P[2 * k + 4]);
        }
        if (s >= 4) {
            const int i = s - 4;  // grid row
            float G[10];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const unsigned g = binom5(hc[i][k], hc[i + 1][k], hc[i + 2][k], hc[i + 3][k], hc[i + 4][k]);
                G[2 * k] = lo_f(g);
                G[2 * k + 1] = hi_f(g);
            }
#pragma unroll
            for (int c = 1; c <= 7; ++c) {
                D[i][c - 1] = G[c + 1] - G[c - 1];
                S[i][c - 1] = fmaf(2.0f, G[c], G[c - 1] + G[c + 1]);
                Gm[i][c - 1] = G[c];
            }
        }
        if (s >= 2) {
            const int r = s - 2;  // raw row of frame t-1
            unsigned P[13];
            row_pairs(reinterpret_cast<const unsigned *>(prv + (int64_t)r * pitch), sh, P);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                hp[r][k] = binom5(P[2 * k + 1], P[2 * k + 2], P[2 * k + 3], P[2 * k + 4], P[2 * k + 5]);
        }
        if (s >= 6) {
            const int w = s - 6;  // window row
            float GP[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned g = binom5(hp[w][k], hp[w + 1][k], hp[w + 2][k], hp[w + 3][k], hp[w + 4][k]);
                GP[2 * k] = lo_f(g);
                GP[2 * k + 1] = hi_f(g);
            }
#pragma unroll
            for (int e = 0; e < 7; ++e) {
                const float ix = fmaf(2.0f, D[w + 1][e], D[w][e] + D[w + 2][e]);
                const float iy = S[w + 2][e] - S[w][e];
                const float it = Gm[w + 1][e] - GP[e];
                a00 = fmaf(ix, ix, a00);
                a01 = fmaf(ix, iy, a01);
                a11 = fmaf(iy, iy, a11);
                b0 = fmaf(ix, it, b0);
                b1 = fmaf(iy, it, b1);
            }
        }
    }
    acc[0] = a00;
    acc[1] = a01;
    acc[2] = a11;
    acc[3] = b0;
    acc[4] = b1;
}

// ---- border points: half a warp, clamped grid ------------------------------------------
//
// The clamped rows and columns within 4 of the point form a grid of nr x nc (<= 9 x 9)
// positions that holds every smoothed value the 7x7 window and its Sobel neighbours read.
// Lane j < nq of the half computes the horizontal Gaussian of frame row q0 + j on the
// grid columns; lane i < nr gathers its five vertical taps by shuffles and holds smoothed
// grid row r0 + i; lane d < 7 accumulates window row d - 3. All values up to the Sobel
// output are integers below 2^24, exact in FP32 and equal to the chain's. Every lane of
// the warp calls this (the shuffles span the warp); the sums land in lane 0 of each half.
__device__ void lk_sums_clamped(const TrackVideo &vd, int frame, int p, float acc[5])
{
    const int lane = threadIdx.x & 15;  // lane within the half-warp
    const int W = vd.W, H = vd.H;
    const int64_t pitch = vd.pitch;
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
    // sum the 7 window rows (fixed order: lanes 0..6 by a tree within the half)
#pragma unroll
    for (int off = 4; off > 0; off >>= 1) {
        a00 += __shfl_down_sync(FULLM, a00, off, 16);
        a01 += __shfl_down_sync(FULLM, a01, off, 16);
        a11 += __shfl_down_sync(FULLM, a11, off, 16);
        b0 += __shfl_down_sync(FULLM, b0, off, 16);
        b1 += __shfl_down_sync(FULLM, b1, off, 16);
    }
    acc[0] = a00;
    acc[1] = a01;
    acc[2] = a11;
    acc[3] = b0;
    acc[4] = b1;
}

// Five blocks per SM (96 registers, a few spilled words) run faster than three without
// spills: the kernel is latency-bound, and the extra warps hide more of it.
__global__ void __launch_bounds__(LK_THREADS, 5) lk_kernel(const TrackVideo one, const TrackVideo *vids, int n_videos,
                                                        int64_t total_frames, int K)
{
    const int lane = threadIdx.x & 31;
    const int64_t gid = (int64_t)blockIdx.x * LK_THREADS + threadIdx.x;
    int64_t gframe;
    int i;
    if (total_frames * K <= 0xffffffffll) {  // 32-bit division when the slots allow
        const unsigned g32 = (unsigned)gid;
        gframe = g32 / (unsigned)K;
        i = (int)(g32 - (unsigned)gframe * (unsigned)K);
    } else {
        gframe = gid / K;
        i = (int)(gid % K);
    }
    const TrackVideo &vd = video_of(one, vids, n_videos, min(gframe, total_frames - 1));
    const int frame = (int)(gframe - vd.frame_begin + vd.first_frame);
    const bool valid = gframe < total_frames && frame > 0 && i < vd.n_points[frame];
    if (!__any_sync(FULLM, valid)) return;  // warp-uniform
    const int W = vd.W, H = vd.H;
    const int64_t o = (int64_t)frame * K + i;
    const int p = valid ? vd.idx[o] : 0;
    const int py = p / W, px = p - py * W;
    const bool interior = valid && px >= 6 && px <= W - 7 && py >= 6 && py <= H - 7;
    if (interior) {
        float s[5];
        lk_sums_interior(vd, frame, px, py, s);
        store_step(vd, o, s[0], s[1], s[2], s[3], s[4]);
    }
    // points with a clamped window: two at a time, one per half-warp; a half without a
    // point repeats the other half's and stores nothing
    unsigned rest = __ballot_sync(FULLM, valid && !interior);
    while (rest) {
        const int la = __ffs(rest) - 1;
        rest &= rest - 1;
        const bool has_b = rest != 0;
        const int lb = has_b ? __ffs(rest) - 1 : la;
        if (has_b) rest &= rest - 1;
        const int src = lane < 16 ? la : lb;
        const long long gf = __shfl_sync(FULLM, (long long)gframe, src);
        const int q = __shfl_sync(FULLM, p, src);
        const long long oq = __shfl_sync(FULLM, (long long)o, src);
        const TrackVideo &vq = video_of(one, vids, n_videos, gf);
        float s[5];
        lk_sums_clamped(vq, (int)(gf - vq.frame_begin + vq.first_frame), q, s);
        if ((lane & 15) == 0 && (lane < 16 || has_b)) store_step(vq, oq, s[0], s[1], s[2], s[3], s[4]);
    }
}

bool select_attr_set[MAX_DEVICES];

}  // namespace

int prepare_select()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return (int)e;
    if (dev >= 0 && dev < MAX_DEVICES && select_attr_set[dev]) return 0;
    e = cudaFuncSetAttribute(select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SEL_DYN_BYTES);
    if (e != cudaSuccess) return (int)e;
    if (dev >= 0 && dev < MAX_DEVICES) select_attr_set[dev] = true;
    return 0;
}

int launch_select(const TrackVideo &one, const TrackVideo *vids, int n, int64_t total_frames, int K, void *stream)
{
    if (K < 1 || K > MAX_K || total_frames > 0x7fffffff) return (int)cudaErrorInvalidValue;
    if (total_frames == 0) return 0;
    const int r = prepare_select();
    if (r) return r;
    select_kernel<<<(unsigned)total_frames, SEL_THREADS, SEL_DYN_BYTES, static_cast<cudaStream_t>(stream)>>>(one, vids,
                                                                                                     n, K);
    return (int)cudaGetLastError();
}

int launch_lk(const TrackVideo &one, const TrackVideo *vids, int n, int64_t total_frames, int K, void *stream)
{
    const int64_t slots = total_frames * K;
    if (slots == 0) return 0;
    const unsigned blocks = (unsigned)((slots + LK_THREADS - 1) / LK_THREADS);
    lk_kernel<<<blocks, LK_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(one, vids, n, total_frames, K);
    return (int)cudaGetLastError();
}

}  // namespace kf
