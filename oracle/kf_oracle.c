/*
 * kf_oracle.c -- plain, slow, FP64 reference of the fused image-kernel chain.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's product path links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header, table or constant with the CUDA path.
 *
 * What it computes is the sequential semantics of a kernel chain (Sec. III): every
 * kernel K_i reads the whole output map of K_{i-1} and writes a whole map of its own,
 * I_out_final = K_n(...K_1(I_in)). Fusion (Sec. V-B, Eq. 2) must reproduce exactly this
 * result, so the oracle is the definition written out, one stage at a time, per frame,
 * in double precision. The concrete stages form the Harris-corner chain whose kinds
 * match Table II: a point conversion, rectangular (stencil) filters, a gradient filter
 * and a threshold, followed by a tracking step that sits across a kernel-to-kernel
 * dependency (Sec. V-A c, Table IV last row).
 *
 * Conventions: a frame is H rows x W columns, x = column (positive right), y = row
 * (positive down). Every stencil clamps its OWN input map to the frame edge
 * (replicates the border pixel).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Stage 1, point operation (Table II row 1, "convert"): f = u8 / 255. */
void kfo_convert(int H, int W, const uint8_t *in, int64_t pitch, double *f)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            f[(int64_t)y * W + x] = (double)in[(int64_t)y * pitch + x] / 255.0;
}

/* Binomial smoothing weights [1 4 6 4 1] / 16 of the Gaussian smoothing filter
 * (Table II row 3, a rectangular operation split into its two separable passes). */
static const double GAUSS5[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};

/* Stage 2: horizontal 5-tap Gaussian, g1(y,x) = sum_k w_k f(y, clamp(x+k)). */
void kfo_gauss_h(int H, int W, const double *in, double *out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double s = 0.0;
            for (int k = -2; k <= 2; ++k)
                s += GAUSS5[k + 2] * in[(int64_t)y * W + clampi(x + k, 0, W - 1)];
            out[(int64_t)y * W + x] = s;
        }
}

/* Stage 3: vertical 5-tap Gaussian, g(y,x) = sum_k w_k g1(clamp(y+k), x). */
void kfo_gauss_v(int H, int W, const double *in, double *out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double s = 0.0;
            for (int k = -2; k <= 2; ++k)
                s += GAUSS5[k + 2] * in[(int64_t)clampi(y + k, 0, H - 1) * W + x];
            out[(int64_t)y * W + x] = s;
        }
}

/* Stage 4, gradient filter (Table II row 4): unnormalised 3x3 Sobel,
 *   Ix = sum_dy s(dy) [g(y+dy, x+1) - g(y+dy, x-1)],  s = (1, 2, 1)
 *   Iy = sum_dx s(dx) [g(y+1, x+dx) - g(y-1, x+dx)]
 * with every index clamped on g. */
void kfo_sobel(int H, int W, const double *g, double *ix, double *iy)
{
    static const double s[3] = {1.0, 2.0, 1.0};
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double gx = 0.0, gy = 0.0;
            for (int d = -1; d <= 1; ++d) {
                int yy = clampi(y + d, 0, H - 1), xx = clampi(x + d, 0, W - 1);
                gx += s[d + 1] * (g[(int64_t)yy * W + clampi(x + 1, 0, W - 1)] -
                                  g[(int64_t)yy * W + clampi(x - 1, 0, W - 1)]);
                gy += s[d + 1] * (g[(int64_t)clampi(y + 1, 0, H - 1) * W + xx] -
                                  g[(int64_t)clampi(y - 1, 0, H - 1) * W + xx]);
            }
            ix[(int64_t)y * W + x] = gx;
            iy[(int64_t)y * W + x] = gy;
        }
}

/* Stage 5, point operation: structure-tensor products. */
void kfo_products(int64_t n, const double *ix, const double *iy, double *pxx, double *pxy,
                  double *pyy)
{
    for (int64_t i = 0; i < n; ++i) {
        pxx[i] = ix[i] * ix[i];
        pxy[i] = ix[i] * iy[i];
        pyy[i] = iy[i] * iy[i];
    }
}

/* Stage 6, rectangular operation: unnormalised 5x5 box sum, all 25 terms, clamped. */
void kfo_box5(int H, int W, const double *in, double *out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double s = 0.0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx)
                    s += in[(int64_t)clampi(y + dy, 0, H - 1) * W + clampi(x + dx, 0, W - 1)];
            out[(int64_t)y * W + x] = s;
        }
}

/* Stage 7, point operation: Harris response R = det(S) - k tr(S)^2. */
void kfo_harris(int64_t n, const double *sxx, const double *sxy, const double *syy, double k,
                double *r)
{
    for (int64_t i = 0; i < n; ++i) {
        double det = sxx[i] * syy[i] - sxy[i] * sxy[i];
        double tr = sxx[i] + syy[i];
        r[i] = det - k * tr * tr;
    }
}

/* Stage 8, threshold (Table II row 5) with 3x3 non-maximum suppression:
 *   mask(p) = R(p) > thr  and  R(p) >= R(q) for every in-frame 8-neighbour q.
 * Returns the number of marked pixels (the per-frame corner count). */
int64_t kfo_nms(int H, int W, const double *r, double thr, uint8_t *mask, int64_t mask_pitch)
{
    int64_t count = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double c = r[(int64_t)y * W + x];
            int keep = c > thr;
            for (int dy = -1; dy <= 1 && keep; ++dy)
                for (int dx = -1; dx <= 1 && keep; ++dx) {
                    int yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    if (r[(int64_t)yy * W + xx] > c) keep = 0;
                }
            mask[(int64_t)y * mask_pitch + x] = (uint8_t)keep;
            count += keep;
        }
    return count;
}

/* Map indices of kfo_chain_frame's optional outputs. */
enum { KFO_F, KFO_G1, KFO_G, KFO_IX, KFO_IY, KFO_PXX, KFO_PXY, KFO_PYY, KFO_SXX, KFO_SXY,
       KFO_SYY, KFO_R, KFO_NMAPS };

/* The whole chain on one frame, unfused, stage by stage.
 * maps: NULL, or KFO_NMAPS pointers (each NULL or H*W doubles) that receive the
 * intermediate maps. mask: H rows at mask_pitch. Returns the corner count. */
int64_t kfo_chain_frame(int H, int W, const uint8_t *in, int64_t pitch, double k, double thr,
                        double **maps, uint8_t *mask, int64_t mask_pitch)
{
    int64_t n = (int64_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * n * KFO_NMAPS);
    if (!buf) return -1;
    double *m[KFO_NMAPS];
    for (int i = 0; i < KFO_NMAPS; ++i) m[i] = buf + (int64_t)i * n;
    kfo_convert(H, W, in, pitch, m[KFO_F]);
    kfo_gauss_h(H, W, m[KFO_F], m[KFO_G1]);
    kfo_gauss_v(H, W, m[KFO_G1], m[KFO_G]);
    kfo_sobel(H, W, m[KFO_G], m[KFO_IX], m[KFO_IY]);
    kfo_products(n, m[KFO_IX], m[KFO_IY], m[KFO_PXX], m[KFO_PXY], m[KFO_PYY]);
    kfo_box5(H, W, m[KFO_PXX], m[KFO_SXX]);
    kfo_box5(H, W, m[KFO_PXY], m[KFO_SXY]);
    kfo_box5(H, W, m[KFO_PYY], m[KFO_SYY]);
    kfo_harris(n, m[KFO_SXX], m[KFO_SXY], m[KFO_SYY], k, m[KFO_R]);
    int64_t count = kfo_nms(H, W, m[KFO_R], thr, mask, mask_pitch);
    if (maps)
        for (int i = 0; i < KFO_NMAPS; ++i)
            if (maps[i]) memcpy(maps[i], m[i], sizeof(double) * n);
    free(buf);
    return count;
}

/* The chain over T frames (frames t at in + t*H*pitch), one frame per OpenMP task.
 * r_out: NULL or T*H*W doubles receiving R. Returns the number of threads used. */
int kfo_chain_volume(int T, int H, int W, const uint8_t *in, int64_t pitch, double k, double thr,
                     uint8_t *masks, int32_t *counts, double *r_out, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int t = 0; t < T; ++t) {
        double *maps[KFO_NMAPS] = {0};
        if (r_out) maps[KFO_R] = r_out + (int64_t)t * H * W;
        counts[t] = (int32_t)kfo_chain_frame(H, W, in + (int64_t)t * H * pitch, pitch, k, thr,
                                             maps, masks + (int64_t)t * H * pitch, pitch);
#ifdef _OPENMP
        if (t == 0) used = omp_get_num_threads();
#endif
    }
    return used;
}

/* ---------------------------------------------------------------------------------
 * Temporal stage: feature selection and Lucas-Kanade tracking.
 *
 * Tracking reads whole-frame results of the chain (the corner set of frame t), so it
 * depends on many blocks of the previous kernel: a kernel-to-kernel dependency
 * (Sec. V-A c) and a separate fusable set, like the Kalman step of Table IV.
 * --------------------------------------------------------------------------------- */

/* The K largest-R corners of a frame (mask set), ties broken by lower raster index.
 * Writes raster indices in descending-R order; returns how many were found (<= K). */
int kfo_select_points(int H, int W, const double *r, const uint8_t *mask, int64_t mask_pitch,
                      int K, int32_t *idx)
{
    int n = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            if (!mask[(int64_t)y * mask_pitch + x]) continue;
            int32_t p = y * W + x;
            double v = r[p];
            /* insertion into the sorted prefix idx[0..n) */
            int pos = n < K ? n : K;
            while (pos > 0) {
                int32_t q = idx[pos - 1];
                if (r[q] > v || (r[q] == v && q < p)) break;
                --pos;
            }
            if (pos >= K) continue;
            int last = n < K ? n : K - 1;
            for (int i = last; i > pos; --i) idx[i] = idx[i - 1];
            idx[pos] = p;
            if (n < K) ++n;
        }
    return n;
}

/* One Lucas-Kanade step per point over a (2*win+1)^2 window, every index clamped:
 *   A = sum [gx^2, gx*gy; gx*gy, gy^2],  b = sum [gx*gt, gy*gt],  (u, v) = -A^{-1} b
 * with gx = Ix/8, gy = Iy/8 (Sobel of the smoothed frame t scaled to unit gain) and
 * gt = g_t - g_{t-1} (difference of the smoothed frames). A window whose determinant
 * satisfies |det| <= 1e-12 (A00 + A11)^2 is reported singular (status 1, u = v = 0). */
void kfo_lk(int H, int W, const double *g_prev, const double *g_cur, const double *ix,
            const double *iy, int n, const int32_t *idx, int win, double *u, double *v,
            int32_t *status)
{
    for (int i = 0; i < n; ++i) {
        int py = idx[i] / W, px = idx[i] % W;
        double a00 = 0, a01 = 0, a11 = 0, b0 = 0, b1 = 0;
        for (int dy = -win; dy <= win; ++dy)
            for (int dx = -win; dx <= win; ++dx) {
                int64_t q = (int64_t)clampi(py + dy, 0, H - 1) * W + clampi(px + dx, 0, W - 1);
                double gx = ix[q] / 8.0, gy = iy[q] / 8.0, gt = g_cur[q] - g_prev[q];
                a00 += gx * gx;
                a01 += gx * gy;
                a11 += gy * gy;
                b0 += gx * gt;
                b1 += gy * gt;
            }
        double det = a00 * a11 - a01 * a01;
        double tr = a00 + a11;
        if (fabs(det) <= 1e-12 * tr * tr) {
            u[i] = 0.0;
            v[i] = 0.0;
            status[i] = 1;
        } else {
            u[i] = -(a11 * b0 - a01 * b1) / det;
            v[i] = -(a00 * b1 - a01 * b0) / det;
            status[i] = 0;
        }
    }
}

/* Tracking of frame pair (t-1, t): runs the chain on frame t, smooths frame t-1,
 * selects up to K corners of frame t and solves one LK step at each. Returns n. */
int kfo_track_pair(int H, int W, const uint8_t *prev, const uint8_t *cur, int64_t pitch, double k,
                   double thr, int K, int win, int32_t *idx, double *u, double *v, int32_t *status)
{
    int64_t n = (int64_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * n * (KFO_NMAPS + 3));
    uint8_t *mask = (uint8_t *)malloc((size_t)n);
    if (!buf || !mask) {
        free(buf);
        free(mask);
        return -1;
    }
    double *maps[KFO_NMAPS];
    for (int i = 0; i < KFO_NMAPS; ++i) maps[i] = buf + (int64_t)i * n;
    double *fp = buf + (int64_t)KFO_NMAPS * n, *g1p = fp + n, *gp = g1p + n;
    kfo_chain_frame(H, W, cur, pitch, k, thr, maps, mask, W);
    kfo_convert(H, W, prev, pitch, fp);
    kfo_gauss_h(H, W, fp, g1p);
    kfo_gauss_v(H, W, g1p, gp);
    int np = kfo_select_points(H, W, maps[KFO_R], mask, W, K, idx);
    kfo_lk(H, W, gp, maps[KFO_G], maps[KFO_IX], maps[KFO_IY], np, idx, win, u, v, status);
    free(buf);
    free(mask);
    return np;
}

/* Tracking over a volume: frame pairs (t-1, t) for t = 1..T-1, one pair per OpenMP
 * task; frame 0 has no points. Outputs are T*K arrays (row t = frame t) and n[T].
 * Returns the number of threads used. */
int kfo_track_volume(int T, int H, int W, const uint8_t *in, int64_t pitch, double k, double thr, int K, int win,
                     int32_t *n, int32_t *idx, double *u, double *v, int32_t *status, int nthreads)
{
    int used = 1;
    if (T > 0) n[0] = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int t = 1; t < T; ++t) {
        const int64_t o = (int64_t)t * K;
        n[t] = kfo_track_pair(H, W, in + (int64_t)(t - 1) * H * pitch, in + (int64_t)t * H * pitch, pitch, k, thr, K, win,
                              idx + o, u + o, v + o, status + o);
#ifdef _OPENMP
        if (t == 1) used = omp_get_num_threads();
#endif
    }
    return used;
}
