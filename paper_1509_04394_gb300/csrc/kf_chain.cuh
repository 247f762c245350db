// kf_chain.cuh -- device code of the Harris-corner chain, one warp per column strip.
//
// A group [A..B] of consecutive stages runs as one fused kernel (Sec. V-B, Eq. 2):
// the group reads the map written by stage A-1 once, keeps every intermediate of
// stages A..B on chip, and writes only the output of stage B. With A == B this is one
// "simple kernel" of the unfused sequence (Sec. III, Eq. 1).
//
// Work decomposition (the output box of Sec. V, Fig. 3, here 1 frame deep): each warp
// owns a strip of 32*KF_C columns (KF_C adjacent columns per lane) and streams down a
// chunk of rows of one frame. The strip carries a halo of the group's accumulated
// horizontal radius on both sides (Alg. 2, with radii summed over the chained stencils);
// the chunk is extended by the accumulated vertical radius above and below.
//   * horizontal stencils read neighbouring columns through warp shuffles;
//   * vertical stencils keep their history in registers: the Gaussian, Sobel and NMS
//     windows as "pass" states ((1,1)^k decompositions, no row rotation), the 5-row box
//     sum as a 5-slot ring addressed by a compile-time phase (the row loop is unrolled
//     by 5 so that no register is ever moved);
//   * warps never wait on each other: no shared memory, no block barrier.
//
// Units. FP32 maps hold integer-scaled values: f' = 255 f, g1' = 4080 g1,
// g' = 65280 g, (Ix', Iy') = 65280 (Ix, Iy), products and box sums 65280^2, R 65280^4.
// Stages 1-4 are then exact in FP32 (all values are integers below 2^24) whatever the
// order of operations, and every later stage is one shared device function, so any
// partition of the chain gives bit-identical results. In the FP16 form the maps of
// stages 1-3 are stored as exact uint16 (scaled units) and the maps of stages 4-7 as
// FP16 in true units (value * scale, rescaled on load); arithmetic stays FP32.
//
// Borders. Every stencil clamps its own input map (replicate). The group's input is
// read with clamped coordinates. Inside the group, a map that feeds a horizontal
// stencil and was itself produced by one is overwritten outside the frame by its edge
// column (shuffle broadcast, only in warps whose strip crosses a frame edge); a vertical
// stage refills its state from its input row 0 and replays its last row past row H-1.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "kf_params.h"

namespace kf {

constexpr unsigned FULL = 0xffffffffu;
constexpr float HARRIS_K = 0.04f;

template <int N> struct Rows { float v[N][C]; };
struct Empty {};

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ float u8_to_float(uint32_t w, int c)
{
    // 0x4B000000 | byte is the float 2^23 + byte; subtracting 2^23 is exact
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (unsigned)c)) - 8388608.0f;
}

__device__ __forceinline__ float pick(const float (&v)[C], int c)
{
    float r = v[0];
#pragma unroll
    for (int j = 1; j < C; ++j) r = (c == j) ? v[j] : r;
    return r;
}

// Columns of this lane outside [0, W) take the value of the edge column (per-stage
// clamp of an on-chip map). Warp-uniform: called only by warps that cross an edge.
template <int N>
__device__ __forceinline__ void fix_edges(Rows<N> &r, int xs, int x0, int W, bool L, bool R)
{
    if (L) {
        const int src = (-xs) / C;  // column 0 sits at register 0 of lane src (xs % C == 0)
#pragma unroll
        for (int m = 0; m < N; ++m) {
            const float e = __shfl_sync(FULL, r.v[m][0], src);
#pragma unroll
            for (int c = 0; c < C; ++c) r.v[m][c] = (x0 + c < 0) ? e : r.v[m][c];
        }
    }
    if (R) {
        const int src = (W - 1 - xs) / C, reg = (W - 1 - xs) % C;
#pragma unroll
        for (int m = 0; m < N; ++m) {
            const float e = __shfl_sync(FULL, pick(r.v[m], reg), src);
#pragma unroll
            for (int c = 0; c < C; ++c) r.v[m][c] = (x0 + c >= W) ? e : r.v[m][c];
        }
    }
}

// Neighbour columns -R..-1 (from the lane to the left) and C..C+R-1 (from the right).
template <int R> struct Halo { float l[R], r[R]; };
template <int R>
__device__ __forceinline__ Halo<R> halo(const float (&v)[C])
{
    Halo<R> h;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        h.l[j] = __shfl_up_sync(FULL, v[C - R + j], 1);
        h.r[j] = __shfl_down_sync(FULL, v[j], 1);
    }
    return h;
}
template <int R>
__device__ __forceinline__ float at(const float (&v)[C], const Halo<R> &h, int c)
{
    return c < 0 ? h.l[R + c] : (c >= C ? h.r[c - C] : v[c]);
}

// ------------------------------------------------------------------ stage arithmetic
// Each function is the only implementation of its stage: fused and unfused kernels
// call the same code, so their results agree bit for bit.

// Stage 2: [1 4 6 4 1] along the row (scaled: no division).
__device__ __forceinline__ void gauss_h(const float (&x)[C], float (&o)[C])
{
    const Halo<2> h = halo<2>(x);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        float t = at<2>(x, h, c - 2) + at<2>(x, h, c + 2);
        t = fmaf(4.0f, at<2>(x, h, c - 1) + at<2>(x, h, c + 1), t);
        o[c] = fmaf(6.0f, x[c], t);
    }
}

// Stage 3: [1 4 6 4 1] down the columns as four (1,1) passes; z[j] = previous value
// at pass level j. Output row = input row - 2.
struct GaussV {
    float z[4][C];
    __device__ __forceinline__ void fill(const float (&x)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) { z[0][c] = x[c]; z[1][c] = 2.0f * x[c]; z[2][c] = 4.0f * x[c]; z[3][c] = 8.0f * x[c]; }
    }
    __device__ __forceinline__ void replay(float (&x)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) x[c] = z[0][c];
    }
    __device__ __forceinline__ void push(const float (&x)[C], float (&o)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float a = x[c] + z[0][c], b = a + z[1][c], d = b + z[2][c];
            o[c] = d + z[3][c];
            z[0][c] = x[c]; z[1][c] = a; z[2][c] = b; z[3][c] = d;
        }
    }
};

// Stage 4: Sobel. Per row: Dx = g(x+1) - g(x-1), Sx = g(x-1) + 2 g(x) + g(x+1);
// then Ix = Dx(r-1) + 2 Dx(r) + Dx(r+1) = (1,1)^2 pass of Dx, Iy = Sx(r+1) - Sx(r-1) =
// (1,-1) then (1,1) pass of Sx. Output row = input row - 1.
struct SobelV {
    float d[2][C];  // Dx passes
    float s[2][C];  // Sx passes
    __device__ __forceinline__ void fill(const float (&dx)[C], const float (&sx)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) { d[0][c] = dx[c]; d[1][c] = 2.0f * dx[c]; s[0][c] = sx[c]; s[1][c] = 0.0f; }
    }
    __device__ __forceinline__ void replay(float (&dx)[C], float (&sx)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) { dx[c] = d[0][c]; sx[c] = s[0][c]; }
    }
    __device__ __forceinline__ void push(const float (&dx)[C], const float (&sx)[C], float (&ix)[C], float (&iy)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float a = dx[c] + d[0][c];
            ix[c] = a + d[1][c];
            d[0][c] = dx[c]; d[1][c] = a;
            const float p = sx[c] - s[0][c];
            iy[c] = p + s[1][c];
            s[0][c] = sx[c]; s[1][c] = p;
        }
    }
};
__device__ __forceinline__ void sobel_h(const float (&g)[C], float (&dx)[C], float (&sx)[C])
{
    const Halo<1> h = halo<1>(g);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float l = at<1>(g, h, c - 1), r = at<1>(g, h, c + 1);
        dx[c] = r - l;
        sx[c] = fmaf(2.0f, g[c], l + r);
    }
}

// Stage 5: structure-tensor products.
__device__ __forceinline__ void products(const Rows<2> &i, Rows<3> &p)
{
#pragma unroll
    for (int c = 0; c < C; ++c) {
        p.v[0][c] = i.v[0][c] * i.v[0][c];
        p.v[1][c] = i.v[0][c] * i.v[1][c];
        p.v[2][c] = i.v[1][c] * i.v[1][c];
    }
}

// Stage 6: 5x5 box sum. Horizontal: the four 5-wide windows of a lane's columns share
// the pair sums A = x-2 + x-1, B = x0 + x1, Cp = x2 + x3, D = x4 + x5 and E = B + Cp
// (11 adds for 4 outputs). Vertical: the five newest rows, oldest first, from a 5-slot
// ring. Output row = input row - 2.
__device__ __forceinline__ void box_h(const float (&x)[C], float (&o)[C])
{
    static_assert(C == 4, "pair-sharing box assumes 4 columns per lane");
    const Halo<2> h = halo<2>(x);
    const float A = h.l[0] + h.l[1], B = x[0] + x[1], Cp = x[2] + x[3], D = h.r[0] + h.r[1];
    const float E = B + Cp;
    o[0] = (A + B) + x[2];
    o[1] = h.l[1] + E;
    o[2] = E + h.r[0];
    o[3] = x[1] + (Cp + D);
}
struct BoxV {
    float ring[5][3][C];
    // slot of the row pushed at phase PH is PH; the row pushed k steps earlier is (PH - k) mod 5
    template <int PH>
    __device__ __forceinline__ void put(const Rows<3> &h)
    {
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int c = 0; c < C; ++c) ring[PH][m][c] = h.v[m][c];
    }
    __device__ __forceinline__ void fill(const Rows<3> &h)
    {
#pragma unroll
        for (int s = 0; s < 5; ++s)
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int c = 0; c < C; ++c) ring[s][m][c] = h.v[m][c];
    }
    template <int PH>
    __device__ __forceinline__ void newest(Rows<3> &h) const
    {
        constexpr int s = (PH + 4) % 5;  // slot written by the previous push
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int c = 0; c < C; ++c) h.v[m][c] = ring[s][m][c];
    }
    template <int PH>
    __device__ __forceinline__ void sum(Rows<3> &o) const
    {
        constexpr int s0 = (PH + 1) % 5, s1 = (PH + 2) % 5, s2 = (PH + 3) % 5, s3 = (PH + 4) % 5;
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int c = 0; c < C; ++c)
                o.v[m][c] = (((ring[s0][m][c] + ring[s1][m][c]) + ring[s2][m][c]) + ring[s3][m][c]) + ring[PH][m][c];
    }
};

// Stage 7: Harris response.
__device__ __forceinline__ void harris(const Rows<3> &s, float (&r)[C])
{
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float sxx = s.v[0][c], sxy = s.v[1][c], syy = s.v[2][c];
        const float det = fmaf(sxx, syy, -(sxy * sxy));
        const float tr = sxx + syy;
        r[c] = fmaf(-HARRIS_K * tr, tr, det);
    }
}

// Stage 8: threshold + 3x3 non-maximum suppression. Horizontal max of 3, then the
// vertical max of 3 as two (max, max) passes; the centre row is one row behind.
struct NmsV {
    float p[2][C];  // max passes
    float rc[C];    // R of the previous row (the centre of the output row)
    __device__ __forceinline__ void fill(const float (&mh)[C], const float (&r)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) { p[0][c] = mh[c]; p[1][c] = mh[c]; rc[c] = r[c]; }
    }
    __device__ __forceinline__ void replay(float (&mh)[C], float (&r)[C])
    {
#pragma unroll
        for (int c = 0; c < C; ++c) { mh[c] = p[0][c]; r[c] = rc[c]; }
    }
    // returns the 4 mask bits of the output row (input row - 1) in bits 0..C-1
    __device__ __forceinline__ unsigned push(const float (&mh)[C], const float (&r)[C], float thr)
    {
        unsigned bits = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float m1 = fmaxf(mh[c], p[0][c]);
            const float m9 = fmaxf(m1, p[1][c]);
            const float centre = rc[c];
            bits |= ((centre > thr) & (centre >= m9)) ? (1u << c) : 0u;
            p[0][c] = mh[c]; p[1][c] = m1; rc[c] = r[c];
        }
        return bits;
    }
};
__device__ __forceinline__ void nms_h(const float (&r)[C], float (&mh)[C])
{
    const Halo<1> h = halo<1>(r);
#pragma unroll
    for (int c = 0; c < C; ++c) mh[c] = fmaxf(fmaxf(at<1>(r, h, c - 1), r[c]), at<1>(r, h, c + 1));
}

// ------------------------------------------------------------------ map I/O
// Every lane reads ONE aligned vector of C elements per map row, at column xb: its own
// columns when they lie in the frame, else the aligned vector holding the edge column.
// Lanes that cross a frame edge then pick, per column, the element of the clamped column.
template <typename TM> struct MapIO;

template <> struct MapIO<float> {
    using Raw = float4;
    __device__ __forceinline__ static Raw load(const void *plane, int64_t off)
    {
        return __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(plane) + off));
    }
    __device__ __forceinline__ static void unpack(const Raw &q, float scale, float (&v)[C])
    {
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ __forceinline__ static void store(void *plane, int64_t off, const float (&v)[C], unsigned in_mask, float scale)
    {
        float *p = static_cast<float *>(plane) + off;
        if (in_mask == (1u << C) - 1) {
            *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) if (in_mask >> c & 1) p[c] = v[c];
        }
    }
};

template <> struct MapIO<__half> {
    using Raw = uint2;
    __device__ __forceinline__ static Raw load(const void *plane, int64_t off)
    {
        return __ldg(reinterpret_cast<const uint2 *>(static_cast<const __half *>(plane) + off));
    }
    __device__ __forceinline__ static void unpack(const Raw &q, float scale, float (&v)[C])
    {
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
        v[0] = a.x * scale; v[1] = a.y * scale; v[2] = b.x * scale; v[3] = b.y * scale;
    }
    __device__ __forceinline__ static void store(void *plane, int64_t off, const float (&v)[C], unsigned in_mask, float scale)
    {
        __half *p = static_cast<__half *>(plane) + off;
        if (in_mask == (1u << C) - 1) {
            const __half2 a = __floats2half2_rn(v[0] * scale, v[1] * scale);
            const __half2 b = __floats2half2_rn(v[2] * scale, v[3] * scale);
            uint2 q;
            q.x = *reinterpret_cast<const uint32_t *>(&a);
            q.y = *reinterpret_cast<const uint32_t *>(&b);
            *reinterpret_cast<uint2 *>(p) = q;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) if (in_mask >> c & 1) p[c] = __float2half_rn(v[c] * scale);
        }
    }
};

// Exact 16-bit integer maps (the integer-valued maps of stages 1-3 in the FP16 form).
template <> struct MapIO<uint16_t> {
    using Raw = uint2;
    __device__ __forceinline__ static Raw load(const void *plane, int64_t off)
    {
        return __ldg(reinterpret_cast<const uint2 *>(static_cast<const uint16_t *>(plane) + off));
    }
    __device__ __forceinline__ static void unpack(const Raw &q, float scale, float (&v)[C])
    {
        v[0] = (float)(q.x & 0xffffu); v[1] = (float)(q.x >> 16); v[2] = (float)(q.y & 0xffffu); v[3] = (float)(q.y >> 16);
    }
    __device__ __forceinline__ static void store(void *plane, int64_t off, const float (&v)[C], unsigned in_mask, float scale)
    {
        uint16_t *p = static_cast<uint16_t *>(plane) + off;
        if (in_mask == (1u << C) - 1) {
            uint2 q;
            q.x = __float2uint_rn(v[0]) | __float2uint_rn(v[1]) << 16;
            q.y = __float2uint_rn(v[2]) | __float2uint_rn(v[3]) << 16;
            *reinterpret_cast<uint2 *>(p) = q;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) if (in_mask >> c & 1) p[c] = (uint16_t)__float2uint_rn(v[c]);
        }
    }
};

// Storage type of the map written by stage k: FP32 maps in the FP32 form; in the FP16
// form exact uint16 for the integer-valued maps of stages 1-3 and FP16 from stage 4 on.
template <int K, bool F16>
using MapT = std::conditional_t<!F16, float, std::conditional_t<(K <= 3), uint16_t, __half>>;

// ------------------------------------------------------------------ the group kernel
template <int A, int B, bool F16>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, MIN_BLOCKS) group_kernel(const GroupParams p)
{
    static_assert(1 <= A && A <= B && B <= 8, "stage range");
    static_assert(C == 4, "map I/O assumes 4 columns per lane");
    constexpr int RXT = sum_rx(A, B);
    constexpr int RYT = sum_ry(A, B);
    constexpr int NIN = map_channels(A - 1);
    constexpr int NOUT = map_channels(B);
    // cumulative vertical delay before stage k
    constexpr int D2 = sum_ry(A, 1), D3 = sum_ry(A, 2), D4 = sum_ry(A, 3), D6 = sum_ry(A, 5), D8 = sum_ry(A, 7);
    constexpr bool HAS3 = A <= 3 && 3 <= B, HAS4 = A <= 4 && 4 <= B, HAS6 = A <= 6 && 6 <= B, HAS8 = A <= 8 && 8 <= B;

    const int lane = threadIdx.x & 31;
    const int64_t job = (int64_t)blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
    if (job >= p.n_jobs) return;  // whole warp leaves together
    const int strip = (int)(job % p.n_strips);
    const int64_t rest = job / p.n_strips;
    const int chunk = (int)(rest % p.n_chunks);
    const int64_t frame = rest / p.n_chunks;
    const int W = p.W, H = p.H;

    const int xs = p.xs0 + strip * p.step;
    const int x0 = xs + C * lane;
    const int xo0 = max(xs + RXT, 0), xo1 = min(xs + RXT + p.step, W);
    const bool edgeL = xs < 0, edgeR = xs + STRIP > W;
    // the one aligned input vector of this lane per row, and the element each column takes
    const int xb = x0 < 0 ? 0 : (x0 >= W ? ((W - 1) & ~(C - 1)) : x0);
    int kc[C];
    unsigned bsel = 0;  // byte selector of the clamped columns (u8 input)
#pragma unroll
    for (int c = 0; c < C; ++c) {
        kc[c] = min(max(x0 + c, 0), W - 1) - xb;
        bsel |= (unsigned)kc[c] << (4 * c);
    }
    const bool lane_inside = (x0 >= 0) && (x0 + C <= W);
    unsigned out_mask = 0;  // which of this lane's columns belong to the strip's output
#pragma unroll
    for (int c = 0; c < C; ++c) out_mask |= (x0 + c >= xo0 && x0 + c < xo1) ? (1u << c) : 0u;

    const int y0 = chunk * p.chunk_rows, y1 = min(y0 + p.chunk_rows, H);
    const int t_begin = max(y0 - RYT, 0), t_end = y1 + RYT;

    // on-chip state of the vertical stages
    std::conditional_t<HAS3, GaussV, Empty> s3{};
    std::conditional_t<HAS4, SobelV, Empty> s4{};
    std::conditional_t<HAS6, BoxV, Empty> s6{};
    std::conditional_t<HAS8, NmsV, Empty> s8{};
    unsigned count = 0;

    const int64_t in_frame = frame * p.in_fstride, out_frame = frame * p.out_fstride;
    auto in_off = [&](int row) { return in_frame + (int64_t)min(max(row, 0), H - 1) * p.in_pitch + xb; };

    // Input rows are prefetched PD = 5 rows ahead into registers (slot = loop phase):
    // u8 frames and single-channel maps. Wider maps are loaded when used.
    using InIO = MapIO<MapT<A - 1, F16>>;
    constexpr bool PREFETCH = (A == 1) || (NIN == 1);
    using RawIn = std::conditional_t<A == 1, uint32_t, typename InIO::Raw>;
    [[maybe_unused]] RawIn q[PREFETCH ? 5 : 1];
    auto load_raw = [&](int row, int m) -> RawIn {
        if constexpr (A == 1) return __ldg(reinterpret_cast<const uint32_t *>(static_cast<const uint8_t *>(p.in[0]) + in_off(row)));
        else return InIO::load(p.in[m], in_off(row));
    };
    if constexpr (PREFETCH) {
#pragma unroll
        for (int k = 0; k < 5; ++k) q[k] = load_raw(t_begin + k, 0);
    }

    auto step = [&](auto phase_tag, int t) {
        [[maybe_unused]] constexpr int PH = decltype(phase_tag)::value;
        const bool border = (t <= RYT) || (t >= H);
        // ---- group input row t (clamped)
        [[maybe_unused]] Rows<1> f;
        [[maybe_unused]] Rows<NIN> in;
        if constexpr (A == 1) {
            const uint32_t w = __byte_perm(q[PH], 0u, bsel);
            q[PH] = load_raw(t + 5, 0);
#pragma unroll
            for (int c = 0; c < C; ++c) f.v[0][c] = u8_to_float(w, c);
        } else {
#pragma unroll
            for (int m = 0; m < NIN; ++m) {
                RawIn raw;
                if constexpr (PREFETCH) {
                    raw = q[PH];
                    q[PH] = load_raw(t + 5, 0);
                } else {
                    raw = load_raw(t, m);
                }
                float v[C];
                InIO::unpack(raw, p.in_scale, v);
                if (lane_inside) {
#pragma unroll
                    for (int c = 0; c < C; ++c) in.v[m][c] = v[c];
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) in.v[m][c] = pick(v, kc[c]);
                }
            }
        }
        // ---- stage 2 (horizontal Gaussian)
        [[maybe_unused]] Rows<1> g1;
        if constexpr (A <= 2 && 2 <= B) {
            if constexpr (A == 1) gauss_h(f.v[0], g1.v[0]);
            else gauss_h(in.v[0], g1.v[0]);
        } else if constexpr (A == 3) {
            g1 = in;
        }
        // ---- stage 3 (vertical Gaussian), input row t - D3
        [[maybe_unused]] Rows<1> g;
        if constexpr (HAS3) {
            if (border) {
                const int i = t - D3;
                if (i == 0) s3.fill(g1.v[0]);
                if (i >= H) s3.replay(g1.v[0]);
            }
            s3.push(g1.v[0], g.v[0]);
        } else if constexpr (A == 4) {
            g = in;
        }
        // ---- stage 4 (Sobel), input row t - D4
        [[maybe_unused]] Rows<2> ixy;
        if constexpr (HAS4) {
            if constexpr (hstencil_before(A, 4))
                if (edgeL | edgeR) fix_edges<1>(g, xs, x0, W, edgeL, edgeR);
            float dx[C], sx[C];
            sobel_h(g.v[0], dx, sx);
            if (border) {
                const int i = t - D4;
                if (i == 0) s4.fill(dx, sx);
                if (i >= H) s4.replay(dx, sx);
            }
            s4.push(dx, sx, ixy.v[0], ixy.v[1]);
        } else if constexpr (A == 5) {
            ixy = in;
        }
        // ---- stage 5 (products)
        [[maybe_unused]] Rows<3> pr;
        if constexpr (A <= 5 && 5 <= B) {
            if constexpr (hstencil_before(A, 6) && HAS6)
                if (edgeL | edgeR) fix_edges<2>(ixy, xs, x0, W, edgeL, edgeR);
            products(ixy, pr);
        } else if constexpr (A == 6) {
            pr = in;
        }
        // ---- stage 6 (box 5x5), input row t - D6
        [[maybe_unused]] Rows<3> sm;
        if constexpr (HAS6) {
            Rows<3> hs;
#pragma unroll
            for (int m = 0; m < 3; ++m) box_h(pr.v[m], hs.v[m]);
            if (border) {
                const int i = t - D6;
                if (i == 0) s6.fill(hs);
                if (i >= H) s6.template newest<PH>(hs);
            }
            s6.template put<PH>(hs);
            s6.template sum<PH>(sm);
        } else if constexpr (A == 7) {
            sm = in;
        }
        // ---- stage 7 (Harris)
        [[maybe_unused]] Rows<1> r;
        if constexpr (A <= 7 && 7 <= B) {
            harris(sm, r.v[0]);
        } else if constexpr (A == 8) {
            r = in;
        }
        // ---- stage 8 (threshold + NMS), input row t - D8
        [[maybe_unused]] unsigned bits = 0;
        if constexpr (HAS8) {
            if constexpr (hstencil_before(A, 8))
                if (edgeL | edgeR) fix_edges<1>(r, xs, x0, W, edgeL, edgeR);
            float mh[C];
            nms_h(r.v[0], mh);
            if (border) {
                const int i = t - D8;
                if (i == 0) s8.fill(mh, r.v[0]);
                if (i >= H) s8.replay(mh, r.v[0]);
            }
            bits = s8.push(mh, r.v[0], p.thr);
        }
        // ---- group output row t - RYT
        const int o = t - RYT;
        if (o >= y0 && o < y1 && out_mask) {
            const int64_t ooff = out_frame + (int64_t)o * p.out_pitch + x0;
            if constexpr (B == 8) {
                const unsigned kept = bits & out_mask;
                uint8_t *mp = static_cast<uint8_t *>(p.out[0]) + ooff;
                if (out_mask == (1u << C) - 1) {
                    *reinterpret_cast<uint32_t *>(mp) = (kept & 1u) | (kept & 2u) << 7 | (kept & 4u) << 14 | (kept & 8u) << 21;
                } else {
#pragma unroll
                    for (int c = 0; c < C; ++c) if (out_mask >> c & 1) mp[c] = (uint8_t)(kept >> c & 1);
                }
                count += __popc(kept);
            } else {
                const Rows<NOUT> *res;
                if constexpr (B == 1) res = &f;
                else if constexpr (B == 2) res = &g1;
                else if constexpr (B == 3) res = &g;
                else if constexpr (B == 4) res = &ixy;
                else if constexpr (B == 5) res = &pr;
                else if constexpr (B == 6) res = &sm;
                else res = &r;
#pragma unroll
                for (int m = 0; m < NOUT; ++m) MapIO<MapT<B, F16>>::store(p.out[m], ooff, res->v[m], out_mask, p.out_scale);
            }
        }
    };

    for (int t = t_begin; t < t_end; t += 5) {
        step(std::integral_constant<int, 0>{}, t);
        if (t + 1 >= t_end) break;
        step(std::integral_constant<int, 1>{}, t + 1);
        if (t + 2 >= t_end) break;
        step(std::integral_constant<int, 2>{}, t + 2);
        if (t + 3 >= t_end) break;
        step(std::integral_constant<int, 3>{}, t + 3);
        if (t + 4 >= t_end) break;
        step(std::integral_constant<int, 4>{}, t + 4);
    }

    if constexpr (B == 8) {
        const unsigned tot = __reduce_add_sync(FULL, count);
        if (lane == 0 && tot) atomicAdd(p.counts + frame, (int)tot);
    }
}

}  // namespace kf
