// kf_params.h -- launch parameters and the stage table shared by host and device code.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the library does not link libcuda)
#include <stdint.h>

#ifdef __CUDACC__
#define KF_HD __host__ __device__
#else
#define KF_HD
#endif

#ifndef KF_C
#define KF_C 4
#endif

namespace kf {

constexpr int C = KF_C;        // columns per lane
constexpr int STRIP = 32 * C;  // columns per warp strip
constexpr int WARPS_PER_BLOCK = 1;  // warps never cooperate: one warp per block
constexpr int MIN_BLOCKS = 16;      // resident blocks per SM the register budget targets
constexpr int MIN_BLOCKS_BOX = 12;  // ... for groups holding the 5-row box ring in registers
constexpr int MIN_BLOCKS_BOX16 = 16; // ... for groups with FP16 inter-stage tiles (the box ring in FP16)
constexpr int NSTAGES = 8;
constexpr int RB = 5;           // rows per TMA stage = rows per unrolled loop block
constexpr int STRIP_ALIGN = 16; // strips start on multiples of 16 columns (16-byte TMA x for u8)
constexpr unsigned WAIT_POLLS = 1u << 22;  // try_wait rounds of a bounded wait before it counts as expired

// Stage table of the Harris chain, 1-based (stage 0 = the u8 frames). One-sided radii
// along columns (rx) and rows (ry), Table I.
KF_HD constexpr int stage_rx(int k) { return k == 2 ? 2 : k == 4 ? 1 : k == 6 ? 2 : k == 8 ? 1 : 0; }
KF_HD constexpr int stage_ry(int k) { return k == 3 ? 2 : k == 4 ? 1 : k == 6 ? 2 : k == 8 ? 1 : 0; }
// channels of the map written by stage k (k = 0: the frames, k = 8: the mask)
KF_HD constexpr int map_channels(int k) { return k == 4 ? 2 : (k == 5 || k == 6) ? 3 : 1; }
KF_HD constexpr int sum_rx(int a, int b) { int s = 0; for (int k = a; k <= b; ++k) s += stage_rx(k); return s; }
KF_HD constexpr int sum_ry(int a, int b) { int s = 0; for (int k = a; k <= b; ++k) s += stage_ry(k); return s; }
// does a stage in [a, k) read horizontal neighbours? (then the input of k needs an edge fix-up)
KF_HD constexpr bool hstencil_before(int a, int k) { for (int j = a; j < k; ++j) if (stage_rx(j) > 0) return true; return false; }

// Capacity of a frame's corner-candidate list for the tracking stage: a quarter of the
// frame (3x3 maxima cannot be denser, except on plateaus), at least 1024.
// keys per frame: a quarter of the pixels (3x3 maxima are at most that dense), at least
// 1024, even (each frame's list starts on 16 bytes)
inline int64_t cand_capacity(int64_t W, int64_t H)
{
    const int64_t q = (W * H + 3) / 4;
    return q < 1024 ? 1024 : q + (q & 1);
}

// Integer scale of the FP32 map written by stage k: scaled = true * map_scale(k).
inline constexpr double map_scale(int k)
{
    return k == 1 ? 255.0 : k == 2 ? 4080.0 : (k == 3 || k == 4) ? 65280.0
         : (k == 5 || k == 6) ? 65280.0 * 65280.0 : k == 7 ? 65280.0 * 65280.0 * 65280.0 * 65280.0 : 1.0;
}

struct GroupParams {
    CUtensorMap tmap[3];      // TMA descriptors of the input planes: {W, H, T}, box {STRIP, RB, 1}
    CUtensorMap tmap_half[3]; // the same planes with box {STRIP/2, RB, 1} (half strips; unused otherwise)
    int *err;                 // device error word (bounded waits that expired)
    const void *in[3];        // input planes (stage A-1 map; u8 frames when A == 1)
    int64_t in_pitch;         // elements between rows
    int64_t in_fstride;       // elements between frames
    void *out[3];             // output planes (u8 mask when B == 8)
    int64_t out_pitch, out_fstride;
    int32_t *counts;          // per-frame corner counts (B == 8), pre-zeroed
    int W, H;                 // frame size
    int xs0, step, n_strips;  // strip s covers input columns [xs0 + s*step, +STRIP)
    int out_off;              // strip s outputs columns [xs + out_off, + step): out_off a multiple of C
    int half_last;            // 1: the last strip is half wide, and one warp runs it for two frames
    int n_lead, n_trail;      // full strips at the frame's left edge (a prefix) and right edge (a suffix)
    int one_full_body;        // 1: interior strips run the edge strips' row loop too (see run_any_job)
    unsigned long long *job_ctr;  // null: block b runs job b; else three counters of jobs taken
                                  // (half-strip, edge, interior; zeroed before the launch) from
                                  // which each block takes its job by the kind its SM prefers
    int sm_split;             // with job_ctr: SMs whose index (scaled to 1024) is below this take
                              // interior jobs first, the others half-strip and edge jobs first
    int T;                    // frames
    int chunk_rows, n_chunks;
    int64_t n_jobs;           // T * n_chunks * (n_strips - half_last) + ceil(T/2) * n_chunks * half_last
    float thr;                // NMS threshold in the scaled units of R
    float in_scale;           // FP16 input maps: scaled value = stored * in_scale
    float out_scale;          // FP16 output maps: stored = scaled value * out_scale
    unsigned wait_polls;      // try_wait rounds a job gives a staged block of input rows (WAIT_POLLS
                              // unless a caller lowered it); the drain of copies in flight after an
                              // expired wait always gets WAIT_POLLS
    // corner candidates for the tracking stage (B == 8, optional): per frame a list of
    // keys (R bits << 32 | ~raster index), cand_cap per frame, cand_count[frame] entries
    unsigned long long *cand;
    int *cand_count;
    int cand_cap;
};

// One video of the tracking stage (by value for a single video, or an array in device
// memory for a batch: frame_begin = the global index of its frame 0 in the batch).
struct TrackVideo {
    const uint8_t *frames;
    int64_t pitch;
    int W, H, T;
    const unsigned long long *cand;  // corner-candidate lists, cand_cap per frame
    const int *cand_count;
    int cand_cap;
    int32_t *n_points, *idx, *status;
    float *u, *v;
    int64_t frame_begin;
    int64_t first_frame;  // one video processed from this frame on (kernel frame 0 = first_frame)
};

// Strip geometry of a group with accumulated horizontal radius rxt: input strips start
// on a multiple of STRIP_ALIGN columns (a legal TMA x for every map type), outputs tile
// the frame exactly. A strip's outputs start out_off = rxt rounded up to whole lanes
// after its first column, so a lane away from the frame's edges outputs all of its
// columns or none.
// The last strip is a half strip (STRIP/2 columns) when that width still reaches the
// frame's last column; a warp then runs the half strips of two frames side by side
// (lanes 0-15 and 16-31), so the mostly idle last strip costs half a warp per frame.
struct StripGeom { int xs0, step, out_off, n_strips, half_last, n_lead, n_trail; };
inline StripGeom strip_geometry(int rxt, int W)
{
    StripGeom g;
    g.xs0 = -((rxt + STRIP_ALIGN - 1) / STRIP_ALIGN) * STRIP_ALIGN;
    g.out_off = (rxt + C - 1) / C * C;
    g.step = ((STRIP - g.out_off - rxt) / STRIP_ALIGN) * STRIP_ALIGN;
    const int o0 = g.xs0 + g.out_off;  // first output column of strip 0 (<= 0)
    g.n_strips = (W - o0 + g.step - 1) / g.step;
    const int xs_last = g.xs0 + (g.n_strips - 1) * g.step;
    g.half_last = (g.n_strips > 1 && xs_last + STRIP / 2 - rxt >= W) ? 1 : 0;
    // full strips whose input box crosses a frame edge: a prefix (xs < 0) and a suffix
    // (xs + STRIP > W); a strip crossing both counts once, in the prefix
    const int F = g.n_strips - g.half_last;
    g.n_lead = (F > 0 && g.xs0 < 0) ? 1 : 0;
    g.n_trail = 0;
    while (g.n_lead + g.n_trail < F && g.xs0 + (F - 1 - g.n_trail) * g.step + STRIP > W) ++g.n_trail;
    return g;
}

#ifdef __CUDACC__
typedef int (*LaunchFn)(const GroupParams &p, unsigned grid, void *stream);
// bytes per element of the map written by 1-based stage k (0 = frames) at a precision
inline int map_elem_bytes(int k, bool f16) { return (k == 0 || k == 8) ? 1 : (f16 ? 2 : 4); }
// f16: 0 = FP32 maps, 1 = 16-bit maps, 2 = 16-bit maps and FP16 inter-stage tiles on chip
LaunchFn launcher_a1(int B, int f16);
LaunchFn launcher_a2(int B, int f16);
LaunchFn launcher_a3(int B, int f16);
LaunchFn launcher_a4(int B, int f16);
LaunchFn launcher_a5(int B, int f16);
LaunchFn launcher_a6(int B, int f16);
LaunchFn launcher_a7(int B, int f16);
LaunchFn launcher_a8(int B, int f16);
int launch_chain_with_candidates(const GroupParams &p, unsigned grid, void *stream);
int launch_chain_with_candidates_tiles(const GroupParams &p, unsigned grid, void *stream);
// tracking kernels over one video (vids == nullptr: `one`) or a table of n videos with
// total_frames frames in all
int prepare_select();  // per-device launch attributes of the selection kernel (before graph capture)
int launch_select(const TrackVideo &one, const TrackVideo *vids, int n, int64_t total_frames, int K, void *stream);
int launch_lk(const TrackVideo &one, const TrackVideo *vids, int n, int64_t total_frames, int K, void *stream);
int launch_batch_chain(const GroupParams *videos, const int64_t *item_begin, int n_videos, unsigned long long *queue,
                       bool cand, unsigned grid, int sm_split, void *stream);
int batch_chain_blocks_per_sm(bool cand);
#endif

}  // namespace kf
