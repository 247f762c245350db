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

// The C = 4 columns of one lane in one row of one map, kept as two FP32 pairs, columns
// (0, 1) and (2, 3). Operations that treat every column alike (vertical stencil passes,
// products, the box's row sums, the Harris response) run as 2-wide FP32 instructions on
// the pairs (add / sub / mul / fma .f32x2: IEEE round-to-nearest per element, so the
// same bits as the scalar operations, at half the issued instructions); horizontal
// stencils read and write single columns, which are halves of the pairs.
struct V4 {
    float2 p[2];
    __device__ __forceinline__ float operator[](int c) const { return (c & 1) ? p[c >> 1].y : p[c >> 1].x; }
    __device__ __forceinline__ float &operator[](int c) { return (c & 1) ? p[c >> 1].y : p[c >> 1].x; }
};
template <int N> struct Rows { V4 v[N]; };
struct Empty {};

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 d;
    asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
        " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}\n"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ V4 add4(const V4 &a, const V4 &b)
{
    V4 r;
    r.p[0] = __fadd2_rn(a.p[0], b.p[0]);
    r.p[1] = __fadd2_rn(a.p[1], b.p[1]);
    return r;
}
__device__ __forceinline__ V4 sub4(const V4 &a, const V4 &b)
{
    V4 r;
    r.p[0] = sub2(a.p[0], b.p[0]);
    r.p[1] = sub2(a.p[1], b.p[1]);
    return r;
}
__device__ __forceinline__ V4 mul4(const V4 &a, const V4 &b)
{
    V4 r;
    r.p[0] = __fmul2_rn(a.p[0], b.p[0]);
    r.p[1] = __fmul2_rn(a.p[1], b.p[1]);
    return r;
}
__device__ __forceinline__ V4 fma4(const V4 &a, const V4 &b, const V4 &c)
{
    V4 r;
    r.p[0] = __ffma2_rn(a.p[0], b.p[0], c.p[0]);
    r.p[1] = __ffma2_rn(a.p[1], b.p[1], c.p[1]);
    return r;
}
__device__ __forceinline__ V4 splat4(float s)
{
    V4 r;
    r.p[0] = r.p[1] = make_float2(s, s);
    return r;
}

// ------------------------------------------------------------------ small helpers
__device__ __forceinline__ float u8_to_float(uint32_t w, int c)
{
    // 0x4B000000 | byte is the float 2^23 + byte; subtracting 2^23 is exact
    return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | (unsigned)c)) - 8388608.0f;
}

__device__ __forceinline__ float pick(const V4 &v, int c)
{
    float r = v[0];
#pragma unroll
    for (int j = 1; j < C; ++j) r = (c == j) ? v[j] : r;
    return r;
}

// The lanes at a frame's edges, in a strip that crosses one: l for the lane holding
// column 0 (always at its register 0: strips start on a multiple of 16 columns), r for the
// lane holding column W-1 (at register rreg). Each stage clamps its own input map at the
// frame's edges; of the lanes outside the frame only these two lanes' stencils would read,
// so the stencils of a map computed on chip take the clamp in the halo of these lanes (the
// edge column's value in place of the neighbour's), and the lanes outside hold values no
// output depends on. The same additions in the same order as a clamped map gives, so the
// results equal those of groups that read the map clamped from memory, bit for bit.
struct EdgeLanes { bool l, r; int rreg; };
constexpr EdgeLanes NO_EDGE{false, false, 0};

// The right-edge lane's columns past W-1 take column W-1's value (when W is not a multiple
// of 4; otherwise column W-1 is a lane's last). Every lane runs it; it changes only that one.
template <int N>
__device__ __forceinline__ void clamp_right_lane(Rows<N> &r, const EdgeLanes &e)
{
#pragma unroll
    for (int m = 0; m < N; ++m) {
        const float x = pick(r.v[m], e.rreg);
#pragma unroll
        for (int c = 0; c < C; ++c) r.v[m][c] = (e.r && c > e.rreg) ? x : r.v[m][c];
    }
}

// Neighbour columns -R..-1 (from the lane to the left) and C..C+R-1 (from the right).
template <int R> struct Halo { float l[R], r[R]; };
template <int R>
__device__ __forceinline__ Halo<R> halo(const V4 &v)
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
__device__ __forceinline__ float at(const V4 &v, const Halo<R> &h, int c)
{
    return c < 0 ? h.l[R + c] : (c >= C ? h.r[c - C] : v[c]);
}

// ------------------------------------------------------------------ stage arithmetic
// Each function is the only implementation of its stage: fused and unfused kernels
// call the same code, so their results agree bit for bit.

// Stage 2: [1 4 6 4 1] along the row (scaled: no division).
__device__ __forceinline__ void gauss_h(const V4 &x, V4 &o)
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
    V4 z[4];
    __device__ __forceinline__ void fill(const V4 &x)
    {
        z[0] = x;
        z[1] = add4(x, x);
        z[2] = add4(z[1], z[1]);
        z[3] = add4(z[2], z[2]);
    }
    __device__ __forceinline__ void replay(V4 &x) { x = z[0]; }
    __device__ __forceinline__ void push(const V4 &x, V4 &o)
    {
        const V4 a = add4(x, z[0]), b = add4(a, z[1]), d = add4(b, z[2]);
        o = add4(d, z[3]);
        z[0] = x;
        z[1] = a;
        z[2] = b;
        z[3] = d;
    }
};

// Stages 2-3 on the frame's bytes, two columns per 32-bit word (16-bit lanes: lo = column
// c, hi = column c + 1). Used by groups that start at the frames and contain both
// Gaussian passes. All Gaussian values are integers (g1' <= 16 * 255, g' <= 65280 < 2^16)
// and every partial sum is at most its total, so no lane carries into the next and the
// results equal the FP32 passes exactly.
__device__ __forceinline__ uint32_t binom5_packed(uint32_t a, uint32_t b, uint32_t c, uint32_t d, uint32_t e)
{
    return (a + e) + ((b + d) << 2) + c * 6u;
}
// g1' of the lane's 4 columns from its bytes w and its neighbours' (L left, R right):
// h01 = (g1'(x0), g1'(x0+1)), h23 = (g1'(x0+2), g1'(x0+3))
__device__ __forceinline__ void gauss_h_packed(uint32_t L, uint32_t w, uint32_t R, uint32_t &h01, uint32_t &h23)
{
    static_assert(C == 4, "packed Gaussian assumes 4 columns per lane");
    const uint32_t pm2 = __byte_perm(L, 0, 0x4342);  // (b-2, b-1)
    const uint32_t p0 = __byte_perm(w, 0, 0x4140);   // (b0, b1)
    const uint32_t p2 = __byte_perm(w, 0, 0x4342);   // (b2, b3)
    const uint32_t p4 = __byte_perm(R, 0, 0x4140);   // (b4, b5)
    const uint32_t pm1 = __funnelshift_r(pm2, p0, 16), p1 = __funnelshift_r(p0, p2, 16), p3 = __funnelshift_r(p2, p4, 16);
    h01 = binom5_packed(pm2, pm1, p0, p1, p2);
    h23 = binom5_packed(p0, p1, p2, p3, p4);
}
// Stage 3 as four (1,1) passes on the packed words (as GaussV, two columns per word).
struct GaussVPacked {
    uint32_t z[4][2];
    __device__ __forceinline__ void fill(const uint32_t (&x)[2])
    {
#pragma unroll
        for (int c = 0; c < 2; ++c) { z[0][c] = x[c]; z[1][c] = x[c] << 1; z[2][c] = x[c] << 2; z[3][c] = x[c] << 3; }
    }
    __device__ __forceinline__ void replay(uint32_t (&x)[2])
    {
#pragma unroll
        for (int c = 0; c < 2; ++c) x[c] = z[0][c];
    }
    __device__ __forceinline__ void push(const uint32_t (&x)[2], uint32_t (&o)[2])
    {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint32_t a = x[c] + z[0][c], b = a + z[1][c], d = b + z[2][c];
            o[c] = d + z[3][c];
            z[0][c] = x[c]; z[1][c] = a; z[2][c] = b; z[3][c] = d;
        }
    }
};
// the two 16-bit lanes of a packed word as an FP32 pair (exact): each lane is placed
// under the exponent of 2^23, and one 2-wide subtraction of 2^23 leaves its value
__device__ __forceinline__ float2 u16x2_to_float2(uint32_t x)
{
    const float2 biased = make_float2(__uint_as_float(__byte_perm(x, 0x4B000000u, 0x7610)),
                                      __uint_as_float(__byte_perm(x, 0x4B000000u, 0x7632)));
    return sub2(biased, make_float2(8388608.0f, 8388608.0f));
}

// Stage 4: Sobel. Per row: Dx = g(x+1) - g(x-1), Sx = g(x-1) + 2 g(x) + g(x+1);
// then Ix = Dx(r-1) + 2 Dx(r) + Dx(r+1) = (1,1)^2 pass of Dx, Iy = Sx(r+1) - Sx(r-1)
// directly from the Sx of two rows before (one subtraction; the values are integers
// below 2^24, so every form gives the same bits). Output row = input row - 1.
struct SobelV {
    V4 d[2];  // Dx passes
    V4 s[2];  // Sx of the previous row and of the one before it
    __device__ __forceinline__ void fill(const V4 &dx, const V4 &sx)
    {
        d[0] = dx;
        d[1] = add4(dx, dx);
        s[0] = sx;
        s[1] = sx;
    }
    __device__ __forceinline__ void replay(V4 &dx, V4 &sx)
    {
        dx = d[0];
        sx = s[0];
    }
    __device__ __forceinline__ void push(const V4 &dx, const V4 &sx, V4 &ix, V4 &iy)
    {
        const V4 a = add4(dx, d[0]);
        ix = add4(a, d[1]);
        d[0] = dx;
        d[1] = a;
        iy = sub4(sx, s[1]);
        s[1] = s[0];
        s[0] = sx;
    }
};
__device__ __forceinline__ void sobel_h(const V4 &g, V4 &dx, V4 &sx, const EdgeLanes &e = NO_EDGE)
{
    Halo<1> h = halo<1>(g);
    h.l[0] = e.l ? g[0] : h.l[0];
    h.r[0] = e.r ? g[C - 1] : h.r[0];
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
    p.v[0] = mul4(i.v[0], i.v[0]);
    p.v[1] = mul4(i.v[0], i.v[1]);
    p.v[2] = mul4(i.v[1], i.v[1]);
}

// Stage 6: 5x5 box sum. Horizontal: the four 5-wide windows of a lane's columns share
// the pair sums A = x-2 + x-1, B = x0 + x1, Cp = x2 + x3, D = x4 + x5 and E = B + Cp;
// A is the left lane's Cp and D the right lane's B (the same two columns added in the
// same order), so they arrive by shuffle with the single columns x-1 and x4 (9 adds
// for 4 outputs). Vertical: each row's sum with the row before it is kept (a 5-slot
// ring addressed by the compile-time loop phase: the row loop is unrolled by 5, so no
// register is ever moved), and the window of rows t-4..t is
// ((r[t-4] + r[t-3]) + (r[t-2] + r[t-1])) + r[t]: 3 adds a value instead of 4, in an
// order fixed by the rows' ages alone, the same in every partition and chunk height.
// Output row = input row - 2.
__device__ __forceinline__ void box_h(const V4 &x, V4 &o, const EdgeLanes &e = NO_EDGE)
{
    static_assert(C == 4, "pair-sharing box assumes 4 columns per lane");
    const float B = x[0] + x[1], Cp = x[2] + x[3];
    float A = __shfl_up_sync(FULL, Cp, 1), D = __shfl_down_sync(FULL, B, 1);
    float xm1 = __shfl_up_sync(FULL, x[3], 1), x4 = __shfl_down_sync(FULL, x[0], 1);
    // at the frame's edges: the clamped neighbours' pair sums and columns
    A = e.l ? x[0] + x[0] : A;
    xm1 = e.l ? x[0] : xm1;
    D = e.r ? x[3] + x[3] : D;
    x4 = e.r ? x[3] : x4;
    const float E = B + Cp;
    o[0] = (A + B) + x[2];
    o[1] = xm1 + E;
    o[2] = E + x4;
    o[3] = x[1] + (Cp + D);
}
struct BoxV {
    V4 pair[5][3];  // slot PH: the row pushed at phase PH plus the row before it
    V4 last[3];     // the newest row
    // the first row of a frame: the rows above it clamp to it
    __device__ __forceinline__ void fill(const Rows<3> &h)
    {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            last[m] = h.v[m];
            const V4 two = add4(h.v[m], h.v[m]);
#pragma unroll
            for (int s = 0; s < 5; ++s) pair[s][m] = two;
        }
    }
    // rows past the frame's end clamp to the last one
    template <int PH>
    __device__ __forceinline__ void newest(Rows<3> &h) const
    {
#pragma unroll
        for (int m = 0; m < 3; ++m) h.v[m] = last[m];
    }
    template <int PH>
    __device__ __forceinline__ void put(const Rows<3> &h)
    {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            pair[PH][m] = add4(last[m], h.v[m]);
            last[m] = h.v[m];
        }
    }
    // after put<PH>: pair (PH + 4) % 5 = r[t-2] + r[t-1], pair (PH + 2) % 5 = r[t-4] + r[t-3]
    template <int PH>
    __device__ __forceinline__ void sum(Rows<3> &o) const
    {
        constexpr int p1 = (PH + 4) % 5, p3 = (PH + 2) % 5;
#pragma unroll
        for (int m = 0; m < 3; ++m) o.v[m] = add4(add4(pair[p3][m], pair[p1][m]), last[m]);
    }
};

// The box's vertical state in the FP16 form: the same ring of row-pair sums held as FP16
// pairs (half the registers), the newest row in FP32. The pair sums are rounded to FP16
// once when formed, the two of a window are added in FP16, and the window's sum is
// accumulated in FP32 with the newest row. Inputs are the products scaled by 2^-32 (an
// exact power of two; see run_job), so every pair sum fits FP16's range.
struct BoxV16 {
    __half2 pair[5][3][2];  // slot PH: the row pushed at phase PH plus the row before it
    V4 last[3];             // the newest row
    __device__ __forceinline__ void fill(const Rows<3> &h)
    {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            last[m] = h.v[m];
            const V4 two = add4(h.v[m], h.v[m]);
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const __half2 t = __float22half2_rn(two.p[k]);
#pragma unroll
                for (int s = 0; s < 5; ++s) pair[s][m][k] = t;
            }
        }
    }
    template <int PH>
    __device__ __forceinline__ void newest(Rows<3> &h) const
    {
#pragma unroll
        for (int m = 0; m < 3; ++m) h.v[m] = last[m];
    }
    template <int PH>
    __device__ __forceinline__ void put(const Rows<3> &h)
    {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const V4 ps = add4(last[m], h.v[m]);
            pair[PH][m][0] = __float22half2_rn(ps.p[0]);
            pair[PH][m][1] = __float22half2_rn(ps.p[1]);
            last[m] = h.v[m];
        }
    }
    template <int PH>
    __device__ __forceinline__ void sum(Rows<3> &o) const
    {
        constexpr int p1 = (PH + 4) % 5, p3 = (PH + 2) % 5;
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
            for (int k = 0; k < 2; ++k)
                o.v[m].p[k] = __fadd2_rn(__half22float2(__hadd2(pair[p3][m][k], pair[p1][m][k])), last[m].p[k]);
    }
};

// Stage 7: Harris response, R = (Sxx Syy - Sxy^2) - k (Sxx + Syy)^2.
__device__ __forceinline__ void harris(const Rows<3> &s, V4 &r)
{
    const V4 det = sub4(mul4(s.v[0], s.v[2]), mul4(s.v[1], s.v[1]));
    const V4 tr = add4(s.v[0], s.v[2]);
    r = fma4(mul4(splat4(-HARRIS_K), tr), tr, det);
}

// Stage 8: threshold + 3x3 non-maximum suppression. Horizontal max of 3, then the
// vertical max of the row and the two before it (one 3-input max); the centre row is one
// row behind.
struct NmsV {
    V4 p[2];  // horizontal maxima of the previous row and of the one before it
    V4 rc;    // R of the previous row (the centre of the output row)
    __device__ __forceinline__ void fill(const V4 &mh, const V4 &r)
    {
        p[0] = mh;
        p[1] = mh;
        rc = r;
    }
    __device__ __forceinline__ void replay(V4 &mh, V4 &r)
    {
        mh = p[0];
        r = rc;
    }
    // returns the 4 mask bits of the output row (input row - 1) in bits 0..C-1, and the
    // response of that row in `centre`
    __device__ __forceinline__ unsigned push(const V4 &mh, const V4 &r, float thr, V4 &centre)
    {
        unsigned bits = 0;
        centre = rc;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float m9 = fmaxf(fmaxf(mh[c], p[0][c]), p[1][c]);
            bits |= ((centre[c] > thr) & (centre[c] >= m9)) ? (1u << c) : 0u;
        }
        p[1] = p[0];
        p[0] = mh;
        rc = r;
        return bits;
    }
};
__device__ __forceinline__ void nms_h(const V4 &r, V4 &mh, const EdgeLanes &e = NO_EDGE)
{
    Halo<1> h = halo<1>(r);
    h.l[0] = e.l ? r[0] : h.l[0];
    h.r[0] = e.r ? r[C - 1] : h.r[0];
#pragma unroll
    for (int c = 0; c < C; ++c) mh[c] = fmaxf(fmaxf(at<1>(r, h, c - 1), r[c]), at<1>(r, h, c + 1));
}

// ------------------------------------------------------------------ TMA staging
// The group's input rows reach shared memory by TMA tensor copies: one copy per channel
// brings RB rows x STRIP columns of one frame; NST such stages form a ring, each with an
// mbarrier. Columns outside the frame and rows past its end arrive as zeros (handled by
// the clamped reads below and by the vertical stages' replay). Every wait is bounded:
// on expiry the kernel records KF_DEVERR_TIMEOUT in the device error word, waits once
// more (bounded, WAIT_POLLS rounds each) for its copies in flight, and leaves.

constexpr int DEVERR_TIMEOUT = 1;
constexpr int DEVERR_OVERFLOW = 2;  // a frame had more corner candidates than cand_cap

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait of at most `polls` try_wait rounds; returns false if they ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned polls = WAIT_POLLS)
{
    for (unsigned i = 0; i < polls; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Reading one staged row: each lane reads its C elements (or, when its columns cross a
// frame edge, the elements of the clamped columns) and converts them to float.
template <typename TM> struct Staged;
template <> struct Staged<uint8_t> {
    // the lane's 4 bytes (clamped columns for a lane at a frame edge) in one word
    __device__ __forceinline__ static uint32_t word(const unsigned char *row, int lane, bool inside, const int (&off)[C])
    {
        if (inside) return *reinterpret_cast<const uint32_t *>(row + C * lane);
        uint32_t w = 0;
#pragma unroll
        for (int c = 0; c < C; ++c) w |= (uint32_t)row[off[c]] << (8 * c);
        return w;
    }
    __device__ __forceinline__ static void read(const unsigned char *row, int lane, bool inside, const int (&off)[C], float, V4 &v)
    {
        const uint32_t w = word(row, lane, inside, off);
#pragma unroll
        for (int c = 0; c < C; ++c) v[c] = u8_to_float(w, c);
    }
};
template <> struct Staged<float> {
    __device__ __forceinline__ static void read(const unsigned char *row, int lane, bool inside, const int (&off)[C], float, V4 &v)
    {
        const float *r = reinterpret_cast<const float *>(row);
        if (inside) {
            const float4 q = reinterpret_cast<const float4 *>(r)[lane];
            v.p[0] = make_float2(q.x, q.y);
            v.p[1] = make_float2(q.z, q.w);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) v[c] = r[off[c]];
        }
    }
};
template <> struct Staged<__half> {
    __device__ __forceinline__ static void read(const unsigned char *row, int lane, bool inside, const int (&off)[C], float scale, V4 &v)
    {
        const __half *r = reinterpret_cast<const __half *>(row);
        if (inside) {
            const uint2 q = reinterpret_cast<const uint2 *>(r)[lane];
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&q.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&q.y));
            v[0] = a.x * scale; v[1] = a.y * scale; v[2] = b.x * scale; v[3] = b.y * scale;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) v[c] = __half2float(r[off[c]]) * scale;
        }
    }
};
template <> struct Staged<uint16_t> {
    __device__ __forceinline__ static void read(const unsigned char *row, int lane, bool inside, const int (&off)[C], float, V4 &v)
    {
        const uint16_t *r = reinterpret_cast<const uint16_t *>(row);
        if (inside) {
            const uint2 q = reinterpret_cast<const uint2 *>(r)[lane];
            v[0] = (float)(q.x & 0xffffu); v[1] = (float)(q.x >> 16); v[2] = (float)(q.y & 0xffffu); v[3] = (float)(q.y >> 16);
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) v[c] = (float)r[off[c]];
        }
    }
};

// ------------------------------------------------------------------ map stores
template <typename TM> struct Store;
template <> struct Store<float> {
    __device__ __forceinline__ static void row(void *plane, int64_t off, const V4 &v, unsigned in_mask, float)
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
template <> struct Store<__half> {
    __device__ __forceinline__ static void row(void *plane, int64_t off, const V4 &v, unsigned in_mask, float scale)
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
template <> struct Store<uint16_t> {
    __device__ __forceinline__ static void row(void *plane, int64_t off, const V4 &v, unsigned in_mask, float)
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

// Storage type of the map written by stage k (k = 0: the u8 frames): FP32 maps in the
// FP32 form; in the FP16 form exact uint16 for the integer-valued maps of stages 1-3 and
// FP16 from stage 4 on.
template <int K, bool F16>
using MapT = std::conditional_t<K == 0, uint8_t, std::conditional_t<!F16, float, std::conditional_t<(K <= 3), uint16_t, __half>>>;

// Shared-memory plan of a group: mbarriers and NST input stages of RB rows.
template <int A, int B, bool F16, bool CAND = false> struct SmemPlan {
    static constexpr int NIN = map_channels(A - 1);
    static constexpr int ELEM = (int)sizeof(MapT<A - 1, F16>);
    static constexpr int ROW_BYTES = STRIP * ELEM;               // one staged row of one channel
    static constexpr int CH_BYTES = RB * ROW_BYTES;              // one stage of one channel
    // a half-strip job stages two frames' half rows as two blocks of RB x ROW_BYTES/2,
    // the second at HALF_OFF (TMA destinations stay on 128 bytes)
    static constexpr int HALF_ROW = ROW_BYTES / 2;
    static constexpr int HALF_OFF = (RB * HALF_ROW + 127) / 128 * 128;
    static constexpr int CH_STRIDE = ((CH_BYTES > HALF_OFF + RB * HALF_ROW ? CH_BYTES : HALF_OFF + RB * HALF_ROW) + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = NIN * CH_STRIDE;
    static constexpr int TX_BYTES = NIN * CH_BYTES;              // bytes one stage's copies bring
    static constexpr int NST = STAGE_BYTES <= 2048 ? 4 : (STAGE_BYTES <= 4096 ? 3 : 2);
    static_assert(RB == 5, "one stage per 5-row block (the box ring period)");
    static constexpr bool HAS6 = A <= 6 && 6 <= B;
    static constexpr int BAR_OFF = 0;
    static constexpr int IN_OFF = 128;
    static constexpr int CAND_OFF = IN_OFF + NST * STAGE_BYTES;
    static constexpr int CAND_LANE = 48;            // buffered corners per lane (entry j of lane l at j * 32 + l)
    static constexpr int CAND_BLOCK = RB * C;       // corners a lane may add in one 5-row block, at most
    static constexpr int RING_OFF = CAND_OFF + (CAND ? CAND_LANE * 32 * 8 : 0);
    static constexpr int RING_BYTES = RB * 32 * C * 4;  // R of the block's output rows, per lane
    static constexpr int BYTES = RING_OFF + (CAND ? RING_BYTES : 0);
};

// ------------------------------------------------------------------ the group kernel
// Job order: the half-strip jobs of the frame pairs (chunk fastest), then the full strips
// at an edge (strip fastest, then chunk, then frame), then the full strips away from the
// frame's edges (likewise). Each kind runs its own instance of the row loop (the interior
// one without any edge handling); kept together, each SM runs one instance at a time,
// which keeps the instruction cache to one loop body (interleaving the half strips with
// the full strips, to find their columns still in L2, measured 40% slower). The longer
// jobs come first, so the launch ends on the short interior jobs, which fill its last
// wave more evenly (the chain 1.30 against 1.38 ms at 200-row tiles with the interior
// strips first).
struct JobPos { int strip, chunk, frame0; bool paired, edge; };
__device__ __forceinline__ JobPos decode_job(const GroupParams &p, int64_t job)
{
    JobPos j;
    const int F = p.n_strips - p.half_last;  // full strips per frame
    const int E = p.n_lead + p.n_trail, I = F - E;
    const int64_t n_pair = p.n_jobs - (int64_t)p.T * p.n_chunks * F;
    const int64_t n_edge = (int64_t)p.T * p.n_chunks * E;
    j.paired = job < n_pair;
    j.edge = job < n_pair + n_edge;
    if (!j.edge) {
        const int64_t q = job - n_pair - n_edge;
        j.strip = p.n_lead + (int)(q % I);
        const int64_t rest = q / I;
        j.chunk = (int)(rest % p.n_chunks);
        j.frame0 = (int)(rest / p.n_chunks);
    } else if (!j.paired) {
        const int64_t q = job - n_pair;
        const int e = (int)(q % E);
        j.strip = e < p.n_lead ? e : F - p.n_trail + (e - p.n_lead);
        const int64_t rest = q / E;
        j.chunk = (int)(rest % p.n_chunks);
        j.frame0 = (int)(rest / p.n_chunks);
    } else {
        const int64_t q = job;
        j.strip = F;
        j.chunk = (int)(q % p.n_chunks);
        j.frame0 = 2 * (int)(q / p.n_chunks);
    }
    return j;
}

template <int A, int B, bool F16, bool CAND, bool PAIRED, bool TILES, bool EDGE>
__device__ __forceinline__ bool run_job(const GroupParams &p, const JobPos &jp, unsigned char *smem, unsigned &kbase,
                                        bool global_desc)
{
    static_assert(!CAND || B == 8, "corner candidates come from the NMS stage");
    static_assert(1 <= A && A <= B && B <= 8, "stage range");
    static_assert(C == 4, "lanes own 4 columns");
    static_assert(WARPS_PER_BLOCK == 1, "one warp per block: the staging ring is per warp");
    using SP = SmemPlan<A, B, F16, CAND>;
    using TIN = MapT<A - 1, F16>;
    constexpr int RXT = sum_rx(A, B);
    constexpr int RYT = sum_ry(A, B);
    constexpr int NIN = SP::NIN;
    constexpr int NOUT = map_channels(B);
    constexpr int D3 = sum_ry(A, 2), D4 = sum_ry(A, 3), D6 = sum_ry(A, 5), D8 = sum_ry(A, 7);
    constexpr bool HAS3 = A <= 3 && 3 <= B, HAS4 = A <= 4 && 4 <= B, HAS6 = SP::HAS6, HAS8 = A <= 8 && 8 <= B;
    // FP16 inter-stage tiles (KF_PREC_F16_TILES) in a group that forms the products on
    // chip and keeps the response on chip (A <= 5, B == 8): the box's ring of row-pair
    // sums in FP16 (BoxV16), on products scaled by 2^-32, so the response and the
    // threshold are scaled by 2^-64 (exact).
    static_assert(!TILES || (F16 && A <= 5 && B == 8), "FP16 tiles: groups forming the products and the response");
    constexpr bool ONCHIP16 = TILES;

    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + SP::BAR_OFF);
    unsigned char *stage_buf = smem + SP::IN_OFF;

    const int lane = threadIdx.x & 31;
    constexpr bool paired = PAIRED;  // == jp.paired
    const int strip = jp.strip, chunk = jp.chunk, frame0 = jp.frame0;
    // a pair's lanes 16-31 run frame0 + 1 (none when T is odd and this is the last pair:
    // those lanes then recompute frame0's half strip and store nothing)
    const int half = paired ? lane >> 4 : 0;
    const int sl = paired ? lane & 15 : lane;  // lane within its strip
    const bool active = frame0 + half < p.T;
    const int frame = active ? frame0 + half : frame0;
    const int W = p.W, H = p.H;
    // per-job copies of the fields the row loop uses: with `p` in global memory the
    // compiler could not keep them in registers across the loop's stores
    const int64_t out_pitch = p.out_pitch;
    const float thr = ONCHIP16 ? p.thr * 0x1p-64f : p.thr, in_scale = p.in_scale, out_scale = p.out_scale;
    void *const out_plane[3] = {p.out[0], p.out[1], p.out[2]};

    const int xs = p.xs0 + strip * p.step;  // multiple of 16 columns: TMA-aligned
    const int x0 = xs + C * sl;
    const int xo0 = max(xs + p.out_off, 0), xo1 = min(xs + p.out_off + p.step, W);
    // EDGE == false: the strip's input box lies inside the frame, so every lane reads its
    // own columns, no on-chip map needs an edge fix-up, and (outputs starting on a lane
    // boundary) each lane outputs all of its columns or none
    static_assert(EDGE || !PAIRED, "half strips are the last strip: an edge");
    const bool edgeL = EDGE && xs < 0, edgeR = EDGE && xs + (paired ? STRIP / 2 : STRIP) > W;
    // the lanes holding columns 0 and W-1, and whether the latter has columns past W-1
    [[maybe_unused]] const EdgeLanes edge{edgeL && x0 == 0, edgeR && x0 <= W - 1 && W - 1 < x0 + C, W - 1 - x0};
    [[maybe_unused]] const bool rpart = edgeR && (W % C) != 0;
    const bool lane_inside = !EDGE || ((x0 >= 0) && (x0 + C <= W));
    int off[C];  // staged-tile offset of each column's clamped source
#pragma unroll
    for (int c = 0; c < C; ++c) off[c] = min(max(x0 + c, 0), W - 1) - xs;
    unsigned out_mask = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) out_mask |= (active && x0 + c >= xo0 && x0 + c < xo1) ? (1u << c) : 0u;
    // staged rows of this lane's strip: base, row pitch, and the lane's position in them
    const int lane_sbase = paired ? half * SP::HALF_OFF : 0;
    const int row_pitch = paired ? SP::HALF_ROW : SP::ROW_BYTES;

    const int y0 = chunk * p.chunk_rows, y1 = min(y0 + p.chunk_rows, H);
    const int t_begin = max(y0 - RYT, 0), t_end = y1 + RYT;
    // stages whose first row lies in the frame; rows of later stages (all past H-1) are
    // replaced by the vertical replay or never stored, so they are neither copied nor awaited
    const int n_stages = min((t_end - t_begin + RB - 1) / RB, (H - t_begin + RB - 1) / RB);

    // ---- staging ring: init barriers, issue the first NST stages
    // stage k of this job is ring stage g = kbase + k: buffer g % NST, mbarrier phase g / NST
    int issued = 0;  // stages issued so far (the same count on every lane)
    auto slot = [&](int k) { return (int)((kbase + (unsigned)k) % SP::NST); };
    auto parity = [&](int k) { return ((kbase + (unsigned)k) / SP::NST) & 1u; };
    const int frame1 = min(frame0 + 1, p.T - 1);
    auto issue = [&](int k) {  // lane 0 only
        uint64_t *bar = bars + slot(k);
        unsigned char *dst = stage_buf + slot(k) * SP::STAGE_BYTES;
        mbar_expect_tx(bar, SP::TX_BYTES);
        if constexpr (!paired) {
#pragma unroll
            for (int m = 0; m < NIN; ++m) tma_load_3d(dst + m * SP::CH_STRIDE, &p.tmap[m], xs, t_begin + k * RB, frame0, bar);
        } else {
#pragma unroll
            for (int m = 0; m < NIN; ++m) {
                tma_load_3d(dst + m * SP::CH_STRIDE, &p.tmap_half[m], xs, t_begin + k * RB, frame0, bar);
                tma_load_3d(dst + m * SP::CH_STRIDE + SP::HALF_OFF, &p.tmap_half[m], xs, t_begin + k * RB, frame1, bar);
            }
        }
    };
    __syncwarp();  // the previous job's lanes have read every stage buffer
    if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (global_desc)  // descriptor written to global memory by the host before the launch
            for (int m = 0; m < NIN; ++m) {
                const CUtensorMap *d = paired ? &p.tmap_half[m] : &p.tmap[m];
                asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(d)) : "memory");
            }
        for (int k = 0; k < SP::NST && k < n_stages; ++k) issue(k);
    }
    issued = min(SP::NST, n_stages);
    __syncwarp();

    // on-chip state of the vertical stages
    // groups that start at the frames and contain both Gaussian passes run them packed
    constexpr bool PACKED = A == 1 && B >= 3 && std::is_same<TIN, uint8_t>::value;
    std::conditional_t<HAS3 && !PACKED, GaussV, Empty> s3{};
    std::conditional_t<PACKED, GaussVPacked, Empty> s3p{};
    std::conditional_t<HAS4, SobelV, Empty> s4{};
    std::conditional_t<HAS6, std::conditional_t<ONCHIP16, BoxV16, BoxV>, Empty> s6{};
    std::conditional_t<HAS8, NmsV, Empty> s8{};
    unsigned count = 0;
    [[maybe_unused]] unsigned long long *cand_buf = reinterpret_cast<unsigned long long *>(smem + SP::CAND_OFF);
    [[maybe_unused]] unsigned cand_n = 0;  // this lane's buffered corners
    // Corners of the current 5-row block: bit 4*PH + c of cand_bits marks column c of the
    // output row of phase PH, whose R values wait in r_ring[PH][lane]; at the end of the
    // block each lane turns its marked corners into keys in its buffer column.
    [[maybe_unused]] float4 *r_ring = reinterpret_cast<float4 *>(smem + SP::RING_OFF);
    [[maybe_unused]] unsigned cand_bits = 0;
    [[maybe_unused]] int cand_o0 = 0;  // output row of phase 0 of the block
    auto emit_candidates = [&]() {
        if constexpr (CAND) {
            while (cand_bits) {  // divergent: lanes with corners only
                const int j = __ffs(cand_bits) - 1;
                cand_bits &= cand_bits - 1;
                const int ph = j >> 2, c = j & 3;
                const float4 rv = r_ring[ph * 32 + lane];
                const float r = c == 0 ? rv.x : c == 1 ? rv.y : c == 2 ? rv.z : rv.w;
                const unsigned raster = (unsigned)((cand_o0 + ph) * W + x0 + c);
                cand_buf[cand_n * 32 + lane] = (unsigned long long)__float_as_uint(r) << 32 | (0xffffffffu - raster);
                ++cand_n;
            }
        }
    };
    // Hand the buffered corners to the frame's list: one global atomic per warp for the
    // space, lane offsets from a warp scan of the lane counts. Done when some lane might
    // not hold another 5-row block, and at the end of the job.
    auto flush_candidates = [&](bool force) {
        if constexpr (CAND) {
            if (__any_sync(FULL, force ? cand_n != 0 : cand_n > (unsigned)(SP::CAND_LANE - SP::CAND_BLOCK))) {
                // scan within each strip's lanes (two 16-lane segments in a half-strip pair)
                const int seg = paired ? 16 : 32;
                unsigned incl = cand_n;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const unsigned y = __shfl_up_sync(FULL, incl, d, seg);
                    if (d < seg && sl >= d) incl += y;
                }
                const unsigned total = __shfl_sync(FULL, incl, seg - 1, seg);
                unsigned pos = 0;
                if (sl == 0 && total) pos = atomicAdd(reinterpret_cast<unsigned *>(p.cand_count) + frame, total);
                pos = __shfl_sync(FULL, pos, 0, seg);
                unsigned long long *dst = p.cand + (int64_t)frame * p.cand_cap;
                const unsigned mine = pos + incl - cand_n;
                for (unsigned j = 0; j < cand_n; ++j)
                    if (mine + j < (unsigned)p.cand_cap) dst[mine + j] = cand_buf[j * 32 + lane];
                if (sl == 0 && pos + total > (unsigned)p.cand_cap) atomicOr(p.err, DEVERR_OVERFLOW);
                cand_n = 0;
            }
        }
    };
    bool failed = false;
    int k_fail = 0;
    const int64_t out_frame = (int64_t)frame * p.out_fstride;

    // One row step at loop phase PH (= row within the staged block, = box ring slot).
    auto step = [&](auto phase_tag, int t, const unsigned char *sbuf) {
        constexpr int PH = decltype(phase_tag)::value;
        const bool border = (t <= RYT) || (t >= H);
        // ---- group input row t (staged; rows past the last copied stage are stale and unused)
        const unsigned char *srow = sbuf + lane_sbase + PH * row_pitch;
        [[maybe_unused]] Rows<NIN> in;
        [[maybe_unused]] Rows<1> f;
        [[maybe_unused]] Rows<1> g1;
        [[maybe_unused]] Rows<1> g;
        if constexpr (PACKED) {
            // ---- stages 2-3 on packed bytes, input row t (stage 3: input row t - D3)
            const uint32_t w = Staged<uint8_t>::word(srow, sl, lane_inside, off);
            const uint32_t L = __shfl_up_sync(FULL, w, 1), R = __shfl_down_sync(FULL, w, 1);
            uint32_t h[2], o[2];
            gauss_h_packed(L, w, R, h[0], h[1]);
            if (border) {
                const int i = t - D3;
                if (i == 0) s3p.fill(h);
                if (i >= H) s3p.replay(h);
            }
            s3p.push(h, o);
            g.v[0].p[0] = u16x2_to_float2(o[0]);
            g.v[0].p[1] = u16x2_to_float2(o[1]);
        } else {
#pragma unroll
        for (int m = 0; m < NIN; ++m) Staged<TIN>::read(srow + m * SP::CH_STRIDE, sl, lane_inside, off, in_scale, in.v[m]);
        if constexpr (A == 1) f = in;
        // ---- stage 2 (horizontal Gaussian)
        if constexpr (A <= 2 && 2 <= B) {
            if constexpr (A == 1) gauss_h(f.v[0], g1.v[0]);
            else gauss_h(in.v[0], g1.v[0]);
        } else if constexpr (A == 3) {
            g1 = in;
        }
        // ---- stage 3 (vertical Gaussian), input row t - D3
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
        }
        // ---- stage 4 (Sobel), input row t - D4
        [[maybe_unused]] Rows<2> ixy;
        if constexpr (HAS4) {
            [[maybe_unused]] EdgeLanes e4 = NO_EDGE;
            if constexpr (EDGE && hstencil_before(A, 4)) {
                if (rpart) clamp_right_lane<1>(g, edge);
                e4 = edge;
            }
            V4 dx, sx;
            sobel_h(g.v[0], dx, sx, e4);
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
            if constexpr (EDGE && hstencil_before(A, 6) && HAS6)
                if (rpart) clamp_right_lane<2>(ixy, edge);
            if constexpr (ONCHIP16) {
#pragma unroll
                for (int m = 0; m < 2; ++m) ixy.v[m] = mul4(ixy.v[m], splat4(0x1p-16f));
            }
            products(ixy, pr);
        } else if constexpr (A == 6) {
            pr = in;
        }
        // ---- stage 6 (box 5x5), input row t - D6
        [[maybe_unused]] Rows<3> sm;
        if constexpr (HAS6) {
            Rows<3> hs;
            [[maybe_unused]] EdgeLanes e6 = NO_EDGE;
            if constexpr (EDGE && hstencil_before(A, 6)) e6 = edge;
#pragma unroll
            for (int m = 0; m < 3; ++m) box_h(pr.v[m], hs.v[m], e6);
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
        [[maybe_unused]] Rows<1> r7;
        if constexpr (A <= 7 && 7 <= B) {
            harris(sm, r7.v[0]);
        } else if constexpr (A == 8) {
            r7 = in;
        }
        // ---- stage 8 (threshold + NMS), input row t - D8
        [[maybe_unused]] unsigned bits = 0;
        [[maybe_unused]] V4 centre;
        if constexpr (HAS8) {
            [[maybe_unused]] EdgeLanes e8 = NO_EDGE;
            if constexpr (EDGE && hstencil_before(A, 8)) {
                if (rpart) clamp_right_lane<1>(r7, edge);
                e8 = edge;
            }
            V4 mh;
            nms_h(r7.v[0], mh, e8);
            if (border) {
                const int i = t - D8;
                if (i == 0) s8.fill(mh, r7.v[0]);
                if (i >= H) s8.replay(mh, r7.v[0]);
            }
            bits = s8.push(mh, r7.v[0], thr, centre);
        }
        // ---- group output row t - RYT
        const int o = t - RYT;
        if constexpr (CAND) {
            // corner candidates of the tracking stage: mark them, keep the row's R
            if constexpr (PH == 0) cand_o0 = o;
            r_ring[PH * 32 + lane] = make_float4(centre[0], centre[1], centre[2], centre[3]);
            if (o >= y0) cand_bits |= (bits & out_mask) << (4 * PH);  // warp-uniform test
        }
        if constexpr (B == 8 && !EDGE) {
            // interior strip: out_mask is 0 (halo lanes) or every column, so the row's mask
            // word is one predicated store per lane, with no divergent block around it
            const bool row_out = o >= y0;  // warp-uniform; o < y1 holds: t < y1 + RYT
            const unsigned kept = row_out ? bits & out_mask : 0u;
            count += __popc(kept);
            uint32_t *mp = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(out_plane[0]) + out_frame +
                                                        (int64_t)o * out_pitch + x0);
            // bit k of `kept` to byte k: kept * (1 + 2^7 + 2^14 + 2^21) puts bit k of the copy
            // shifted by 7j at 8j when k == j, and elsewhere at k + 7j, never a multiple of 8
            // for k != j (|k - j| < 7)
            if (row_out && out_mask) *mp = (kept * 0x00204081u) & 0x01010101u;
        } else if (o >= y0 && out_mask) {  // o < y1 holds: t < y1 + RYT
            const int64_t ooff = out_frame + (int64_t)o * out_pitch + x0;
            if constexpr (B == 8) {
                const unsigned kept = bits & out_mask;
                uint8_t *mp = static_cast<uint8_t *>(out_plane[0]) + ooff;
                if (out_mask == (1u << C) - 1) {
                    *reinterpret_cast<uint32_t *>(mp) = (kept * 0x00204081u) & 0x01010101u;
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
                else res = &r7;
                // an interior lane that outputs anything outputs all of its columns
                const unsigned st_mask = EDGE ? out_mask : (1u << C) - 1;
#pragma unroll
                for (int m = 0; m < NOUT; ++m) Store<MapT<B, F16>>::row(out_plane[m], ooff, res->v[m], st_mask, out_scale);
            }
        }
    };

    // Blocks of RB = 5 rows: wait for the block's stage, run the 5 unrolled row steps,
    // then hand the stage buffer back to TMA for block k + NST.
    using P0 = std::integral_constant<int, 0>;
    using P1 = std::integral_constant<int, 1>;
    using P2 = std::integral_constant<int, 2>;
    using P3 = std::integral_constant<int, 3>;
    using P4 = std::integral_constant<int, 4>;

#pragma unroll 1
    for (int k = 0, t = t_begin; t < t_end; ++k, t += RB) {
        if (k < n_stages) {
            const bool ok = __all_sync(FULL, mbar_wait(bars + slot(k), parity(k), p.wait_polls));
            if (!ok) {  // warp-uniform
                failed = true;
                k_fail = k;
                break;
            }
        }
        const unsigned char *sbuf = stage_buf + slot(k) * SP::STAGE_BYTES;
        step(P0{}, t, sbuf);
        if (t + 1 >= t_end) break;
        step(P1{}, t + 1, sbuf);
        if (t + 2 >= t_end) break;
        step(P2{}, t + 2, sbuf);
        if (t + 3 >= t_end) break;
        step(P3{}, t + 3, sbuf);
        if (t + 4 >= t_end) break;
        step(P4{}, t + 4, sbuf);
        emit_candidates();
        flush_candidates(false);
        if (k + SP::NST < n_stages) {
            __syncwarp();  // every lane has read the stage
            if (lane == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(k + SP::NST);
            }
            issued = k + SP::NST + 1;
        }
    }

    if (failed) {
        // record, then give the copies still in flight a bounded chance to land
        if (lane == 0) atomicOr(p.err, DEVERR_TIMEOUT);
        for (int k = k_fail; k < issued; ++k) mbar_wait(bars + slot(k), parity(k), WAIT_POLLS);
        return false;
    }
    emit_candidates();       // a block cut short by the end of the job
    flush_candidates(true);  // what is left at the end of the job
    if constexpr (B == 8) {
        // per strip: one 32-lane strip, or the two 16-lane halves of a pair
        unsigned tot = count;
#pragma unroll
        for (int d = 8; d > 0; d >>= 1) tot += __shfl_xor_sync(FULL, tot, d);
        tot += paired ? 0u : __shfl_xor_sync(FULL, tot, 16);
        if (sl == 0 && tot) atomicAdd(p.counts + frame, (int)tot);
    }
    kbase += (unsigned)n_stages;
    return true;
}

template <int NST>
__device__ __forceinline__ void init_ring(unsigned char *smem)
{
    if ((threadIdx.x & 31) == 0) {
        uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
#pragma unroll
        for (int s = 0; s < NST; ++s) mbar_init(bars + s, 1);
        mbar_fence_init();
    }
    __syncwarp();
}

// a job of either kind: full strip, or a pair of half strips (warp-uniform choice).
// Interior strips have a row loop of their own, without edge handling, which a long launch
// runs for most of its time alone (its queue is kind-major). A launch of about one wave
// runs every kind at once instead, and warps of different row loops on one SM then miss
// the instruction cache (the stall on instruction fetch rose from 1.3 to 6.2 per issue);
// with p.one_full_body interior strips take the edge strips' loop, which is correct for
// them too: two loop bodies instead of three.
template <int A, int B, bool F16, bool CAND, bool TILES = false>
__device__ __forceinline__ bool run_any_job(const GroupParams &p, int64_t job, unsigned char *smem, unsigned &kbase,
                                            bool global_desc)
{
    const JobPos jp = decode_job(p, job);
    if (!jp.edge && !p.one_full_body)
        return run_job<A, B, F16, CAND, false, TILES, false>(p, jp, smem, kbase, global_desc);
    if (!jp.paired) return run_job<A, B, F16, CAND, false, TILES, true>(p, jp, smem, kbase, global_desc);
    return run_job<A, B, F16, CAND, true, TILES, true>(p, jp, smem, kbase, global_desc);
}

// The job of this block when jobs are taken by SM (p.job_ctr): the SMs below p.sm_split
// (of 1024, over %nsmid) take interior jobs first, the others half-strip jobs, then edge
// jobs, so each SM runs one instance of the row loop for most of the launch instead of
// all three kinds meeting on every SM as the queue passes from one kind to the next
// (measured on the 1000-frame chain with corner lists: 1.36 against 1.39 ms at 200-row
// tiles, 1.36 against 1.47 at 267). A kind whose counter has run out is passed over for
// the next; the blocks are as many as the jobs, so every block finds one (a block passes
// over a kind only once all its jobs are taken, and a block that passed over all three
// would mean every job was taken by the others). -1 if not.
__device__ __forceinline__ int64_t pick_job(const GroupParams &p)
{
    long long job = -1;
    if ((threadIdx.x & 31) == 0) {
        unsigned sm, nsm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsm));
        const bool inner_first = (unsigned long long)sm * 1024ull < (unsigned long long)p.sm_split * nsm;
        const int F = p.n_strips - p.half_last;
        const int64_t n_pair = p.n_jobs - (int64_t)p.T * p.n_chunks * F;
        const int64_t n_edge = (int64_t)p.T * p.n_chunks * (p.n_lead + p.n_trail);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (job >= 0) break;
            const int k = inner_first ? 2 - i : i;  // 0 half strips, 1 edge, 2 interior
            const int64_t base = k == 0 ? 0 : k == 1 ? n_pair : n_pair + n_edge;
            const int64_t cnt = k == 0 ? n_pair : k == 1 ? n_edge : p.n_jobs - n_pair - n_edge;
            if (cnt <= 0) continue;
            const unsigned long long t = atomicAdd(p.job_ctr + k, 1ull);
            if ((int64_t)t < cnt) job = (long long)(base + (int64_t)t);
        }
    }
    return __shfl_sync(FULL, job, 0);
}

// One job per block (one warp): the launch's blocks enumerate the jobs, or take them by SM.
template <int A, int B, bool F16, bool CAND = false, bool TILES = false>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, TILES ? MIN_BLOCKS_BOX16 : (A <= 6 && 6 <= B) ? MIN_BLOCKS_BOX : MIN_BLOCKS) group_kernel(const __grid_constant__ GroupParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if ((int64_t)blockIdx.x >= p.n_jobs) return;
    const int64_t job = p.job_ctr ? pick_job(p) : (int64_t)blockIdx.x;
    if (job < 0) return;
    init_ring<SmemPlan<A, B, F16, CAND>::NST>(smem);
    unsigned kbase = 0;
    run_any_job<A, B, F16, CAND, TILES>(p, job, smem, kbase, false);
}

// Persistent batch over many videos (the fully fused chain): each resident warp pops
// jobs from one global counter until the queue is empty; a job's queue segment (binary
// search over item_begin) names its video and the kind of its strip, and the job runs
// with that video's descriptor.
template <bool CAND>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, MIN_BLOCKS_BOX) batch_kernel(const GroupParams *videos, const int64_t *item_begin,
                                                                                      int n_videos, unsigned long long *queue,
                                                                                      int sm_split)
{
    extern __shared__ __align__(128) unsigned char smem[];
    init_ring<SmemPlan<1, 8, false, CAND>::NST>(smem);
    // The queue is kind-major: every video's half-strip jobs, then every video's
    // edge-strip jobs, then every video's interior-strip jobs (segment s = kind * n +
    // video, item_begin[s] its first item), so the launch runs one instance of the row
    // loop at a time, as a single video's launch does, and ends on the shortest jobs.
    // Each kind has its own counter (queue[kind]), and a warp takes its next job from the
    // kind its SM prefers while that kind lasts, as a single video's launch does
    // (pick_job): SMs below sm_split (of 1024) prefer interior strips.
    const int n_seg = 3 * n_videos;
    unsigned kbase = 0;
    bool inner_first = false;
    if ((threadIdx.x & 31) == 0) {
        unsigned sm, nsm;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
        asm volatile("mov.u32 %0, %%nsmid;" : "=r"(nsm));
        inner_first = (unsigned long long)sm * 1024ull < (unsigned long long)sm_split * nsm;
    }
    for (;;) {
        long long item = -1;
        if ((threadIdx.x & 31) == 0) {
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if (item >= 0) break;
                const int k = inner_first ? 2 - i : i;  // 0 half strips, 1 edge, 2 interior
                const int64_t b0 = item_begin[k * n_videos], b1 = item_begin[(k + 1) * n_videos];
                if (b1 <= b0) continue;
                const unsigned long long t = atomicAdd(queue + k, 1ull);
                if ((int64_t)t < b1 - b0) item = (long long)(b0 + (int64_t)t);
            }
        }
        item = __shfl_sync(FULL, item, 0);
        if (item < 0) break;
        int lo = 0, hi = n_seg - 1;  // last s with item_begin[s] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_begin[mid] <= (int64_t)item) lo = mid; else hi = mid - 1;
        }
        const int kind = lo / n_videos, v = lo - kind * n_videos;
        const GroupParams &p = videos[v];
        // the video's job number in decode_job's order (half strips, edge, interior)
        int64_t job = (int64_t)item - item_begin[lo];
        if (kind > 0) {
            const int F = p.n_strips - p.half_last;
            job += p.n_jobs - (int64_t)p.T * p.n_chunks * F;  // the half-strip jobs
            if (kind > 1) job += (int64_t)p.T * p.n_chunks * (p.n_lead + p.n_trail);  // the edge jobs
        }
        if (!run_any_job<1, 8, false, CAND>(p, job, smem, kbase, true)) break;
    }
}

}  // namespace kf
