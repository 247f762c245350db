/*
 * kfuse.h -- C ABI of the fused image-kernel chain library (libkfuse.so).
 *
 * The calls follow the paper's statement of the problem:
 *   1. declare the kernels of a chain with their data-access radii (Sec. IV, Table I;
 *      Alg. 2 reads (2dx+1) x (2dy+1) x dt pixels per thread) -- kf_add_stage;
 *   2. choose the partition into contiguous fused groups that minimises the predicted
 *      global<->on-chip traffic, each kernel covered exactly once (Sec. VI, Fig. 5;
 *      traffic of Sec. VI-D) -- kf_plan, kf_enumerate, kf_partition_traffic;
 *   3. run the fused groups in sequence over the video volume, each group reading its
 *      input box once and keeping its intermediates on chip (Sec. V-B, Eq. 2; Alg. 1)
 *      -- kf_run, kf_run_group.
 *
 * Conventions (all calls):
 *   - Every call returns a kf_status; nothing is thrown across the ABI.
 *   - Pointers named "device" are CUDA device pointers owned by the caller; the library
 *     never allocates, frees or keeps them past the call.
 *   - Calls that take `stream` (a cudaStream_t, NULL = legacy default stream) are
 *     asynchronous: they enqueue work and return. Launch failures are reported as
 *     KF_ECUDA; kf_last_cuda_error() gives the CUDA error code.
 *   - A frame is H rows x W columns; x = column (positive right), y = row (positive
 *     down). Volumes hold T frames back to back.
 *   - Bad arguments are rejected with KF_EINVAL before anything is enqueued.
 *   - Workspace sizes and runs take volumes of W, H in 1..2^30, T in 0..2^31-1 and at
 *     most 2^46 pixels in all (a batch: its videos together); larger ones are KF_EINVAL,
 *     so that no byte count overflows 64 bits. Calls state tighter bounds where they
 *     have them (e.g. W * H below 2^31 for tracking).
 *   - One context per host thread; a context is not thread-safe.
 *   - A call that works on a context's GPU makes that device current for its duration
 *     and gives the caller's current device back before it returns.
 */
#ifndef KFUSE_H
#define KFUSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KF_VERSION_MAJOR 1
#define KF_VERSION_MINOR 0
#define KF_MAX_STAGES 24

typedef enum kf_status {
    KF_OK = 0,
    KF_EINVAL = 1,        /* invalid argument: null pointer, shape, pitch, alignment, range */
    KF_ENOMEM = 2,        /* host allocation failed, or workspace smaller than required    */
    KF_ECUDA = 3,         /* a CUDA runtime call failed; see kf_last_cuda_error()          */
    KF_ESMEM = 4,         /* a group exceeds the on-chip limit (restriction c, Sec. VII)    */
    KF_EUNSUPPORTED = 5,  /* the declared chain can be planned but not executed            */
    KF_ESTATE = 6,        /* call not valid for this context (e.g. run on a host-only ctx) */
    KF_ETIMEOUT = 7       /* a bounded device-side wait expired                            */
} kf_status;

/* Stage kinds. KF_STAGE_CUSTOM stages can only be planned (radii and byte counts come
 * from the descriptor); the eight Harris stages can also be executed, in this order: */
typedef enum kf_stage_kind {
    KF_STAGE_CUSTOM = 0,
    KF_STAGE_CONVERT = 1,  /* f = u8/255                 point,         r = (0,0,0)  */
    KF_STAGE_GAUSS_H = 2,  /* [1 4 6 4 1]/16 along x     rectangular,   r = (2,0,0)  */
    KF_STAGE_GAUSS_V = 3,  /* [1 4 6 4 1]/16 along y     rectangular,   r = (0,2,0)  */
    KF_STAGE_SOBEL = 4,    /* (Ix, Iy), 3x3 Sobel        gradient,      r = (1,1,0)  */
    KF_STAGE_PRODUCTS = 5, /* Ix^2, IxIy, Iy^2           point,         r = (0,0,0)  */
    KF_STAGE_BOX5 = 6,     /* 5x5 sum of each product    rectangular,   r = (2,2,0)  */
    KF_STAGE_HARRIS = 7,   /* R = det - 0.04 tr^2        point,         r = (0,0,0)  */
    KF_STAGE_NMS = 8       /* R > 1e-5 and 3x3 maximum   threshold,     r = (1,1,0)  */
} kf_stage_kind;

typedef enum kf_precision {
    KF_PREC_F32 = 0, /* FP32 maps between groups, FP32 arithmetic                         */
    KF_PREC_F16 = 1, /* 16-bit maps between groups: exact uint16 for the integer-valued
                        maps of stages 1-3, FP16 (true units) for stages 4-7; FP32
                        arithmetic on chip                                               */
    KF_PREC_F16_TILES = 2 /* 16-bit maps as KF_PREC_F16, and FP16 inter-stage tiles on chip
                        in the groups that form the structure-tensor products and keep the
                        response on chip (first stage <= 5, last stage 8): the box's row-pair
                        sums are held in FP16 (products scaled by 2^-32), the window sums
                        accumulated in FP32. Error within the FP16 tolerance (2e-3 of the
                        frame's largest response); results differ from the FP32 groups'   */
} kf_precision;

typedef enum kf_dtype { KF_DT_U8 = 0, KF_DT_F32 = 1, KF_DT_F16 = 2, KF_DT_U16 = 3 } kf_dtype;

/* A kernel of the chain (Table I). Radii are one-sided: the stage reads columns
 * x-rx..x+rx, rows y-ry..y+ry and frames t-rt..t. Byte counts are per pixel over all
 * channels of the stage's input and output maps; 0 means "the builtin default" for the
 * eight Harris kinds at the context precision. */
typedef struct kf_stage_desc {
    int kind;       /* kf_stage_kind                         */
    int rx, ry, rt; /* one-sided radii                       */
    double in_bytes, out_bytes;
} kf_stage_desc;

/* Volume size and the output box x*y*t of one thread block (Sec. V, Fig. 3) that the
 * traffic model assumes. box_* = 0 selects the executor's own tile: x = the output
 * width of a warp strip of the fully fused chain (112 columns), y = the chunk height
 * (kf_set_chunk_rows), t = 1. */
typedef struct kf_geometry {
    int64_t W, H, T;
    int64_t box_x, box_y, box_t;
} kf_geometry;

/* Input video: T frames of H rows of W uint8 pixels, row y of frame t at
 * frames + (t*H + y)*pitch. pitch >= W and a multiple of 16 bytes; frames 16-byte
 * aligned. Device memory, read only. */
typedef struct kf_video {
    const uint8_t *frames;
    int64_t W, H, T;
    int64_t pitch;
} kf_video;

/* Output of the chain. mask: device, same layout as the frames with mask_pitch (a
 * multiple of 16 bytes); pixel = 1 for a corner, 0 otherwise; columns >= W untouched.
 * counts: device, T int32, overwritten with the number of corners of each frame. */
typedef struct kf_corners {
    uint8_t *mask;
    int64_t mask_pitch;
    int32_t *counts;
} kf_corners;

/* A map between groups: `channels` planes (1..3) of T frames x H rows, row y of frame t
 * of plane c at plane[c] + (t*frame_stride + y*pitch) elements. pitch and frame_stride
 * in elements, each a multiple of 16 bytes; planes 16-byte aligned. U8 for the frames and
 * the mask; for the maps of stages 1..7 F32 (KF_PREC_F32), or U16 for stages 1-3 and F16
 * for stages 4-7 (KF_PREC_F16). kf_map_scale gives their units. */
typedef struct kf_map {
    void *plane[3];
    int channels;
    int dtype; /* kf_dtype */
    int64_t pitch, frame_stride;
} kf_map;

typedef struct kf_ctx kf_ctx;

/* Message for a status code (static string). */
const char *kf_status_str(kf_status s);
/* CUDA error code of the last KF_ECUDA on this context (0 if none). */
int kf_last_cuda_error(const kf_ctx *ctx);
kf_status kf_version(int *major, int *minor);

/* Create a context on CUDA device `device` (allocates the context's 4-byte device error
 * word with that device current; the caller's current device is restored), or a
 * host-only planning context when device < 0 (no CUDA call is ever made by it). */
kf_status kf_create(int device, kf_ctx **out);
kf_status kf_destroy(kf_ctx *ctx);

/* Synchronise the device, then return and clear the context's device error word: 0 if
 * every bounded device-side wait of the kernels launched since the last call completed,
 * KF_DEVERR_TIMEOUT if a wait for staged input rows expired (that job's output rows
 * are then incomplete). */
#define KF_DEVERR_TIMEOUT 1
kf_status kf_device_error(kf_ctx *ctx, int *code);

/* KF_PREC_F32 (default), KF_PREC_F16 or KF_PREC_F16_TILES. Changes the builtin byte
 * counts and the dtype of the maps kf_run keeps in the workspace (16-bit for both FP16
 * forms), and with KF_PREC_F16_TILES the on-chip tiles of the groups it names. */
kf_status kf_set_precision(kf_ctx *ctx, int precision);
/* Rows per warp job of the executor (default 200, >= 1). */
kf_status kf_set_chunk_rows(kf_ctx *ctx, int rows);
/* Rows per warp job of the chain launches kf_track_host makes, one per chunk of frames
 * (>= 1), or 0 (default): the kf_set_chunk_rows height. Results do not depend on it.
 * KF_EINVAL if rows < 0. */
kf_status kf_set_host_chunk_rows(kf_ctx *ctx, int rows);
/* Bound of the device-side waits for staged input (the chain's TMA row blocks and the
 * spatio-temporal box's frame copies): the number of mbarrier try_wait rounds a block
 * gives one wait before it records KF_DEVERR_TIMEOUT in the context's error word,
 * waits (bounded, 2^22 rounds each) for the copies it still has in flight, and ends
 * its job, leaving that job's outputs incomplete. Default 2^22 (far beyond any copy's
 * latency). A caller may lower it; 0 makes every such wait expire at once, which shows
 * the timeout path end to end without a fault: kf_device_error then reports
 * KF_DEVERR_TIMEOUT, and calls made after restoring the default give full results.
 * Kernels launched afterwards take the value; a batch (kf_batch_create) keeps the value
 * it was created with. */
kf_status kf_set_wait_polls(kf_ctx *ctx, unsigned polls);

/* Declare the next kernel of the chain (Sec. IV). Returns its 0-based index in *id.
 * KF_EINVAL if the chain already holds KF_MAX_STAGES stages or radii are negative. */
kf_status kf_add_stage(kf_ctx *ctx, const kf_stage_desc *desc, int *id);
/* Declare the eight Harris stages in order (KF_EINVAL if stages were declared before). */
kf_status kf_add_harris_chain(kf_ctx *ctx);
/* Number of stages declared so far in *n (KF_EINVAL for a NULL argument). */
kf_status kf_num_stages(const kf_ctx *ctx, int *n);

/* ------------------------------------------------------------------ planning (host) */
/* A partition is a cut mask: bit i set = a group boundary between stage i and i+1
 * (0-based). 0 = everything fused into one kernel; (1<<(n-1))-1 = no fusion. */

/* Traffic of one fused group [first, last] (0-based, inclusive) in bytes (Sec. VI-D):
 * boxes * ((x+2Rx)(y+2Ry)(t+Rt) in_bytes(first) + x*y*t out_bytes(last)), with
 * boxes = W*H*T/(x*y*t) and R* the SUM of the group's radii. */
kf_status kf_group_traffic(const kf_ctx *ctx, int first, int last, const kf_geometry *g, double *bytes);
/* On-chip bytes the group holds per box: (x+2Rx)(t+Rt) * sum_k (2 ry_k + 1) in_bytes_k. */
kf_status kf_group_onchip(const kf_ctx *ctx, int first, int last, const kf_geometry *g, double *bytes);
/* Total traffic of a partition. KF_EINVAL if the mask has bits at or above n-1. */
kf_status kf_partition_traffic(const kf_ctx *ctx, uint32_t cuts, const kf_geometry *g, double *bytes);
/* The partition of minimum traffic among those whose every group holds at most
 * onchip_limit bytes (restriction c); exact, by dynamic programming over the n-1 cut
 * points (the set-partition model of Fig. 5 restricted to contiguous groups).
 * KF_ESMEM if no partition is feasible. */
kf_status kf_plan(const kf_ctx *ctx, const kf_geometry *g, double onchip_limit, uint32_t *cuts, double *bytes);
/* All 2^(n-1) cut masks in increasing order; *n_out = 2^(n-1) even when cap is smaller
 * (only the first cap are written). */
kf_status kf_enumerate(const kf_ctx *ctx, uint32_t *buf, int64_t cap, int64_t *n_out);

/* ------------------------------------------------------------------ execution (device) */
/* Factor that turns a stored value of the map written by 0-based stage `stage` into the
 * chain's true units (true = stored * factor). FP32 maps hold integer-scaled values
 * (f*255, g1*4080, g*65280, I*65280, products and sums *65280^2, R*65280^4), which keeps
 * stages 1-4 exact; in the FP16 form the uint16 maps of stages 1-3 hold the same scaled
 * integers and the FP16 maps of stages 4-7 hold true units (factor 1). */
kf_status kf_map_scale(const kf_ctx *ctx, int stage, double *factor);

/* Bytes of device workspace kf_run needs for partition `cuts` on a T x H x W volume:
 * the maps at the cut points, double buffered, with rows padded to 16 bytes. */
kf_status kf_workspace_bytes(const kf_ctx *ctx, uint32_t cuts, int64_t W, int64_t H, int64_t T, size_t *bytes);

/* Run the declared Harris chain with partition `cuts` on `stream`: one fused kernel per
 * group, in chain order. Requires a device context whose chain is exactly the eight
 * builtin stages (else KF_EUNSUPPORTED). workspace: device, >= kf_workspace_bytes, 256-byte
 * aligned (may be NULL when cuts == 0). Writes out->mask and out->counts. With T == 0
 * nothing is enqueued and the pointers are not inspected. */
kf_status kf_run(kf_ctx *ctx, uint32_t cuts, const kf_video *video, const kf_corners *out,
                 void *workspace, size_t workspace_bytes, void *stream);

/* Run one fused group [first, last] (0-based stages of the builtin chain) from map `in`
 * (the output of stage first-1; the U8 frames when first == 0) into map `out` (the
 * output of stage last; the U8 mask when last == 7, then `counts` (T int32, device) is
 * overwritten with per-frame corner counts). Map dtypes must match the context
 * precision. */
kf_status kf_run_group(kf_ctx *ctx, int first, int last, const kf_map *in, const kf_map *out,
                       int64_t W, int64_t H, int64_t T, int32_t *counts, void *stream);

/* ------------------------------------------------------------------ tracking */
/* The temporal stages after the chain. Selecting a frame's strongest corners needs the
 * whole frame, a kernel-to-kernel dependency (Sec. V-A c) that closes the chain's
 * fusable set, as the Kalman step does in Table IV; tracking forms the next set.
 * Per frame t >= 1: the K corners of frame t with the largest R (ties: lower raster
 * index first), and one Lucas-Kanade step per corner against frame t-1 over a 7x7
 * window (every index clamped): A = sum [gx^2, gx gy; gx gy, gy^2], b = sum [gx gt, gy gt],
 * (u, v) = -A^-1 b, gx, gy = Sobel of the smoothed frame t divided by 8, gt = smoothed
 * frame t minus smoothed frame t-1. Window sums in FP32; determinant and solve in FP64;
 * a window with |det| <= 1e-12 (A00 + A11)^2 is reported singular (u = v = 0). */
typedef struct kf_tracks {
    int32_t K;          /* points per frame, 1..1024                                      */
    int32_t *n_points;  /* device, T: points of frame t (min(K, corners); 0 for t = 0)   */
    int32_t *idx;       /* device, T*K: raster index y*W + x, strongest first             */
    float *u, *v;       /* device, T*K: motion from frame t-1 to t in px/frame, x / y     */
    int32_t *status;    /* device, T*K: 0 solved, 1 singular window                       */
} kf_tracks;

/* Workspace of kf_track: per frame a corner-candidate list of max(1024, ceil(W*H/4))
 * 8-byte entries and a counter, and the chain launch's job counters (so two calls in
 * flight at once need two workspaces). A frame with more corners than that sets
 * KF_DEVERR_OVERFLOW in the device error word (its selection then covers only the
 * listed corners). */
#define KF_DEVERR_OVERFLOW 2
kf_status kf_track_workspace_bytes(const kf_ctx *ctx, int64_t W, int64_t H, int64_t T, size_t *bytes);
/* The whole hot path on `stream`: the fully fused chain (mask, counts as kf_run with
 * cuts == 0), then corner selection and tracking into `tracks`. workspace: device,
 * >= kf_track_workspace_bytes, 256-byte aligned. W*H must be below 2^31. */
kf_status kf_track(kf_ctx *ctx, const kf_video *video, const kf_corners *out, const kf_tracks *tracks,
                   void *workspace, size_t workspace_bytes, void *stream);
/* kf_track from host memory to host memory, pipelined (the paper has no counterpart; a
 * serving path for video that arrives in host memory). The frames go in and the results
 * come back in chunks of `chunk` frames (the first and the last a quarter of that) on
 * the context's own streams (one copy-in, three compute used in turn, one copy-out at the
 * lowest priority, one for the tracking at the highest): the copy in of chunk k, the
 * chains of the chunks before it and the copies out of earlier ones overlap; selection
 * and LK run over the frames up to the first chunk end at or past T/2 once those
 * chains are done, and over the rest after the last chain. A chunk's chain is a short
 * launch (50 frames of 800x600 about one wave) whose last wave the next chunks' launches
 * fill; kf_set_host_chunk_rows sets its tile height. host_video / host_out /
 * host_tracks: host buffers of the same shapes and pitches as the device ones (page-locked, e.g. cudaHostAlloc, for the copies to be
 * asynchronous; pageable memory still gives correct results, without overlap). video /
 * out / tracks / workspace: device buffers as for kf_track (video holds all T frames; LK
 * of a chunk's first frame reads the previous chunk's last). mask_format: KF_MASK_BYTES,
 * host_out->mask like the device mask (same mask_pitch); or KF_MASK_BITS, the mask
 * packed for transfer, 8 pixels a byte: frame f's pixel (y, x), i = y W + x, is bit i % 8
 * of byte f * host_out->mask_pitch + i / 8 (mask_pitch = bytes per frame, >= ceil(W H /
 * 8), a multiple of 16; bits past W H up to the next 4-byte boundary are 0, the rest of
 * each frame's stride is not written). With KF_MASK_BITS the chunks are packed
 * on the device into a staging ring the context owns (3 chunks of min(chunk, T) packed frames,
 * allocated on first use and grown when a call needs more) and copied out from there;
 * the device mask is written as well. Asynchronous: `stream` waits for the
 * last copy out, and the copies start after the work queued on `stream` before the call;
 * the host buffers must stay valid until then. */
#define KF_MASK_BYTES 0
#define KF_MASK_BITS 1
kf_status kf_track_host(kf_ctx *ctx, const kf_video *host_video, const kf_corners *host_out,
                        const kf_tracks *host_tracks, const kf_video *video, const kf_corners *out,
                        const kf_tracks *tracks, void *workspace, size_t workspace_bytes, int64_t chunk, int mask_format,
                        void *stream);

/* ------------------------------------------------------------------ batches */
/* Many independent videos of different sizes and lengths through the fully fused chain
 * (and optionally the tracking stages) as ONE persistent kernel launch: every resident
 * warp pops jobs (video, frame, row chunk, column strip) from one global queue until it
 * is empty, so long and short videos share the GPU without a per-video launch. The
 * launch, the counter resets and the batched selection and LK kernels are captured once
 * into a CUDA graph by kf_batch_create and replayed by kf_batch_run. FP32 contexts only
 * (full fusion has no maps between groups). The chunk height is the context's
 * (kf_set_chunk_rows / kf_tune_chunk_rows) at creation, or chosen per video with
 * kf_batch_create_ex. */
typedef struct kf_batch kf_batch;
/* Workspace of a batch of n videos; track_K = 0 without tracking, else the points per
 * frame (1..1024). */
kf_status kf_batch_workspace_bytes(const kf_ctx *ctx, const kf_video *videos, int n, int track_K, size_t *bytes);
/* videos, outs: n entries; tracks: NULL, or n entries with the same K. The workspace
 * (>= kf_batch_workspace_bytes, 256-byte aligned) and every buffer named here must stay
 * allocated and in place while the batch exists: the graph refers to them. Synchronous
 * (copies the per-video descriptors into the workspace, captures and instantiates the
 * graph). */
kf_status kf_batch_create(kf_ctx *ctx, const kf_video *videos, const kf_corners *outs, const kf_tracks *tracks, int n,
                          void *workspace, size_t workspace_bytes, kf_batch **out);
/* kf_batch_create with the tile shape chosen per video and the launch's size chosen:
 * chunk_rows (NULL, or n entries >= 1) gives each video's rows per job (its tile height;
 * the tile width is the warp strip, 112 output columns, or a half strip for the last
 * one); warps_per_sm (0 = as many as fit) caps the persistent launch at that many
 * resident warps per SM. The queue hands out jobs longest first (rows per job, then jobs
 * per video), so the launch ends on its shortest jobs. kf_batch_create is this call with
 * NULL and 0. */
kf_status kf_batch_create_ex(kf_ctx *ctx, const kf_video *videos, const kf_corners *outs, const kf_tracks *tracks, int n,
                             const int *chunk_rows, int warps_per_sm, void *workspace, size_t workspace_bytes,
                             kf_batch **out);
/* Enqueue one run of the batch on `stream` (asynchronous): every video's mask, counts and,
 * if requested, tracks are rewritten. */
kf_status kf_batch_run(kf_batch *batch, void *stream);
/* Free the batch's executable graph (a run still in flight completes first) and its
 * host state; the caller's workspace and buffers are not touched. NULL is a no-op. */
kf_status kf_batch_destroy(kf_batch *batch);

/* Autotuner of the executor's tile height: runs the fully fused chain on `video` once
 * per candidate chunk height (after one warm-up), `reps` times each, times them with CUDA
 * events on `stream`, keeps the fastest in the context and returns it (and its time in
 * ms when best_ms is not NULL). Synchronous. */
kf_status kf_tune_chunk_rows(kf_ctx *ctx, const kf_video *video, const kf_corners *out, const int *candidates, int n,
                             int reps, void *stream, int *best_rows, float *best_ms);
/* The same autotuner on the whole hot path: times kf_track (the chain with corner lists,
 * selection, LK; same arguments) per candidate height, keeps the fastest in the context.
 * The chain's launch with corner lists takes its jobs by SM kind, so its best height can
 * differ from the plain chain's. Synchronous. */
kf_status kf_tune_track_rows(kf_ctx *ctx, const kf_video *video, const kf_corners *out, const kf_tracks *tracks,
                             void *workspace, size_t workspace_bytes, const int *candidates, int n, int reps,
                             void *stream, int *best_rows, float *best_ms);
/* The partition of least MEASURED time: the exhaustive check that judges the traffic
 * model's choice (Sec. VI, Fig. 5, against the measured No / Two / Full Fusion of
 * Sec. VII-B). Runs each candidate cut mask (`cands`, n_cand of them; all 2^(n-1) when
 * cands == NULL) on the video once untimed and then `reps` times, each run bracketed by
 * a CUDA event pair on `stream`, and returns the cut mask of the least median time in
 * *best_cuts (the first one on ties), that time in *best_ms and, when ms_all is not
 * NULL, every candidate's median time (n entries, in candidate order). `ws` (device,
 * 256-byte aligned) must hold kf_workspace_bytes of every candidate (KF_ENOMEM before
 * any work otherwise). Synchronises `stream`; the outputs hold the last run's results.
 * The context keeps its precision: with KF_PREC_F16 the cut maps are 16-bit. */
kf_status kf_plan_measured(kf_ctx *ctx, const kf_video *video, const kf_corners *out, void *ws, size_t ws_bytes,
                           const uint32_t *cands, int n_cand, int reps, void *stream, uint32_t *best_cuts, float *best_ms,
                           float *ms_all);

/* ------------------------------------------------------------------ kernel DAGs */
/* Arbitrary DAGs of generic image kernels (Sec. III's chain generalised to one or two
 * inputs per kernel), for planning with learned costs. Node 0 is the frame (u8 / 255);
 * stage i (1-based) writes node i and reads in1 (and in2) < i. Every stencil clamps its
 * own input. Kinds:                                                                     */
#define KF_G_AFFINE 1  /* y = a x + b                                                    */
#define KF_G_ABS 2     /* y = |x|                                                        */
#define KF_G_PRODUCT 3 /* y = min(max(x1 x2, -16), 16)                                   */
#define KF_G_STENCIL 4 /* separable binomial smoothing, radius 0..3: C(2r, r+k) / 4^r    */
#define KF_G_MAX3 5    /* 3x3 maximum                                                    */
#define KF_DAG_MAX_STAGES 24
#define KF_NFEAT 12
typedef struct kf_gstage {
    int kind, in1, in2, radius;
    float a, b;
} kf_gstage;
typedef struct kf_dag kf_dag;
/* The DAG's output is its last node. Groups are contiguous ranges of the stage order; a
 * group runs as one fused kernel (Alg. 1: its input boxes copied to shared memory once,
 * stages on shared-memory tiles, only the maps later groups read are stored). */
kf_status kf_dag_create(kf_ctx *ctx, const kf_gstage *stages, int n, kf_dag **out);
/* Free a DAG made by kf_dag_create (host memory only). NULL is a no-op. */
kf_status kf_dag_destroy(kf_dag *dag);
/* For group [first, last] (0-based stages): KF_NFEAT cost-model features (stages,
 * stencils, largest input halo, summed radii, bytes in and out per pixel, shared memory
 * per block in KiB, peak live tiles, arithmetic per pixel with halo recompute, external
 * inputs, stored outputs, log of the volume), its on-chip bytes per block and its
 * traffic (Sec. VI-D over the executor's 32 x 16 tile). Any pointer may be NULL. */
kf_status kf_dag_group_info(const kf_dag *dag, int first, int last, int64_t W, int64_t H, int64_t T, float *features,
                            double *onchip_bytes, double *traffic_bytes);
/* Exact minimum-cost partition for per-group costs group_cost[g] (n(n+1)/2 entries, group
 * [a, b] at a*n - a(a-1)/2 + (b-a), 0-based; negative or infinite = infeasible), by the
 * same dynamic program as kf_plan. */
kf_status kf_dag_plan(const kf_dag *dag, const double *group_cost, uint32_t *cuts, double *cost);
/* Workspace of kf_dag_run / kf_dag_time_groups: one float map per node. */
kf_status kf_dag_workspace_bytes(const kf_dag *dag, int64_t W, int64_t H, int64_t T, size_t *bytes);
/* Run partition `cuts` on `stream`; the output node's map goes to `out` (T x H rows of
 * out_pitch floats). KF_ESMEM if a group exceeds the on-chip limit. T <= 65535. */
kf_status kf_dag_run(kf_dag *dag, uint32_t cuts, const kf_video *video, float *out, int64_t out_pitch, void *workspace,
                     size_t workspace_bytes, void *stream);
/* Measure every candidate group: runs the DAG unfused once, then each of the n(n+1)/2
 * groups (one warm-up, `reps` timed launches, CUDA events on `stream`); ms[g] = mean
 * time, -1 for infeasible groups. Synchronous. */
kf_status kf_dag_time_groups(kf_dag *dag, const kf_video *video, float *out, int64_t out_pitch, void *workspace,
                             size_t workspace_bytes, int reps, void *stream, float *ms);

/* Plans beyond contiguous partitions: recompute instead of store (the ordering
 * restriction of Sec. VII (a) relaxed for nodes that are cheaper to recompute than to
 * read back). A plan is (cuts, inline_mask): the contiguous ranges of `cuts`, and the
 * inlined nodes (bit j-1 = node j; never the output node n) that are never stored -- every
 * group that needs an inlined node computes it itself, with its inlined inputs, from the
 * stored maps and the frame. A group thus computes its range (less inlined nodes only
 * later groups need) plus the inlined nodes it needs, and stores the output and every
 * range node not inlined from which a path through inlined nodes reaches a later stage.
 * With inline_mask 0 this is the contiguous partition of kf_dag_run. */
#define KF_DAG_EXACT_INLINE 12
/* Sec. VI-D traffic of a plan over the executor's 32 x 16 tile (as kf_dag_group_info)
 * and the largest shared-memory bytes per block of its groups (max_onchip may be NULL). */
kf_status kf_dag_xplan_traffic(const kf_dag *dag, uint32_t cuts, uint32_t inline_mask, int64_t W, int64_t H, int64_t T,
                               double *bytes, double *max_onchip);
/* The cheapest plan whose groups fit onchip_limit bytes of shared memory per block (<= 0
 * or above the executor's 200 KiB: the executor's limit). Cost of a group: its traffic
 * (model NULL), or the learned model's predicted time from the features of the group's
 * own program (`model` a context whose cost model is trained or set; else KF_ESTATE).
 * Search: for every inline set the exact dynamic program over cut points (a group's cost
 * depends only on its range and the inline set); over inline sets exhaustively when the
 * DAG has at most KF_DAG_EXACT_INLINE + 1 stages, else by hill climbing over single-node
 * toggles from the best contiguous partition (never worse than it). *cost: bytes or ms.
 * KF_ESMEM if nothing fits. */
kf_status kf_dag_plan_recompute(const kf_dag *dag, int64_t W, int64_t H, int64_t T, double onchip_limit, kf_ctx *model,
                                uint32_t *cuts, uint32_t *inline_mask, double *cost);
/* Measure groups of plans with inlined nodes, for training the learned model on them:
 * groups[3 g .. 3 g + 2] = (first, last, inline_mask) of group g (0-based stages). Runs
 * the DAG unfused once (so every stored map exists), then each group (one warm-up, `reps`
 * timed launches, CUDA events on `stream`): ms[g] = mean time, -1 if it exceeds the
 * on-chip limit; features (NULL or count x KF_NFEAT) = the group's cost-model features.
 * Synchronous. */
kf_status kf_dag_time_xgroups(kf_dag *dag, const kf_video *video, float *out, int64_t out_pitch, void *workspace,
                              size_t workspace_bytes, const int32_t *groups, int count, int reps, void *stream,
                              float *ms, float *features);
/* Run plan (cuts, inline_mask) on `stream`, like kf_dag_run. */
kf_status kf_dag_run_x(kf_dag *dag, uint32_t cuts, uint32_t inline_mask, const kf_video *video, float *out,
                       int64_t out_pitch, void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ learned cost model */
/* A 3-layer MLP (width 64, ReLU, FP32) predicting a fused group's runtime from its
 * KF_NFEAT features, in place of the execution-time estimate C_i of the partition model
 * (Sec. VI, Fig. 5). Inputs: log1p(features) standardised by the training set; output:
 * standardised log(ms). Parameters: W1 (64 x KF_NFEAT, row = unit), b1, W2 (64 x 64),
 * b2, w3 (64), b3. The model lives in the context. */
#define KF_MLP_NPARAMS (64 * KF_NFEAT + 64 + 64 * 64 + 64 + 64 + 1)
/* Train on n measured groups (features n x KF_NFEAT, runtimes ms > 0) with `steps`
 * full-batch Adam steps on the GPU (He initialisation from `seed`; deterministic). Device
 * memory for the data and the optimiser is allocated for the call and freed before it
 * returns. Returns the final mean squared error on the standardised log-runtimes. */
kf_status kf_costmodel_train(kf_ctx *ctx, const float *features, const float *ms, int n, int steps, float lr,
                             unsigned seed, float *final_loss);
/* Predicted runtime (ms) of n groups from their feature rows (host arrays, n x
 * KF_NFEAT in, n out); KF_ESTATE before training or set. On a context with a GPU the
 * network runs in the library's inference kernel (one thread per row, parameters in
 * shared memory; device memory is allocated for the call's duration); a planning
 * context without a GPU (device < 0) evaluates it on the host. The recompute planner
 * (kf_dag_plan_recompute) evaluates its one-group-at-a-time queries on the host. */
kf_status kf_costmodel_predict(kf_ctx *ctx, const float *features, int n, float *ms);
/* The raw network (no standardisation) at `params` for n input rows x (n x KF_NFEAT),
 * outputs y (n), computed by the inference kernel on the context's GPU (host arrays;
 * KF_ESTATE on a context without a GPU). */
kf_status kf_costmodel_forward(kf_ctx *ctx, const float *params, const float *x, int n, float *y);
/* Loss and gradient of the raw network (no standardisation) at `params` for inputs x
 * (n x KF_NFEAT) and targets y, computed by the training kernels on the GPU. */
kf_status kf_costmodel_grad(kf_ctx *ctx, const float *params, const float *x, const float *y, int n, float *grad,
                            float *loss);
/* Save / load: params (KF_MLP_NPARAMS), norm = feature means (KF_NFEAT), feature
 * deviations (KF_NFEAT), log-runtime mean, log-runtime deviation. */
kf_status kf_costmodel_get(kf_ctx *ctx, float *params, float *norm);
kf_status kf_costmodel_set(kf_ctx *ctx, const float *params, const float *norm);

/* ------------------------------------------------------------------ no-allocation run */
/* kf_run with the workspace in a fixed array that the library itself holds on every GPU
 * that loads it (KF_STATIC_WORKSPACE_BYTES per GPU, kept until the process exits). The
 * paper has no counterpart; this call exists for callers that cannot call cudaMalloc or
 * hand over device memory: a plug-in running inside a host framework that owns all
 * device allocations, or a real-time pipeline whose memory footprint is fixed at start-up.
 * The caller still passes the video and the output buffers, as for kf_run.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine.
 *   - The first call on a device looks up the device address of that device's array
 *     (cudaGetSymbolAddress, with the context's device current); make that first call
 *     before any stream capture.
 *   - KF_ENOMEM when kf_workspace_bytes(cuts, W, H, T) exceeds KF_STATIC_WORKSPACE_BYTES:
 *     split the volume into fewer frames per call (cuts == 0 needs no workspace).
 *   - All calls on a device share the one array and it keeps the last call's contents
 *     (the chain overwrites every map it reads, so nothing needs clearing). Calls whose
 *     kernels overlap on the GPU (other streams, other host threads) race on it:
 *     serialise them.
 *   - The looked-up address is kept for the life of the process. A caller that resets
 *     a device (cudaDeviceReset) after its first call on it must not call this entry
 *     point on that device again: the kept address belonged to the destroyed context.
 *   - Like every entry point, the call leaves the caller's current device as it found it. */
#define KF_STATIC_WORKSPACE_BYTES (64u << 20)
kf_status kf_run_static(kf_ctx *ctx, uint32_t cuts, const kf_video *video, const kf_corners *out, void *stream);

/* ------------------------------------------------------------------ the paper's own chain */
/* The chain of Sec. VII (Table II / Table IV), as one more fusable set: K1 convert RGBA to
 * gray, K2 IIR filter (a point operation over frames), K3 Gaussian smoothing, K4 gradient
 * filter, K5 threshold computation; then K6, a Kalman filter over feature positions,
 * after the kernel-to-kernel dependency. The paper names the steps, not their formulas;
 * the readings (all in the library's scaled units, true value = scaled / scale):
 *   K1  Y' = 77 R + 150 G + 29 B                        (scale 65280; alpha ignored)
 *   K2  y'_0 = Y'_0, y'_t = y'_{t-1} + (Y'_t - y'_{t-1}) / 4   (FP32; scale 65280)
 *   K3  G' = sum w(dy) w(dx) y'(clamp(p + d)), w = [1 2 1]     (scale 16 * 65280)
 *   K4  M' = |sum s(dy) (G'(y+dy,x+1) - G'(y+dy,x-1))| + |same transposed|, s = [1 2 1],
 *       indices clamped on G'                                  (scale 16 * 65280)
 *   K5  mask = M' > 0.25 * 16 * 65280 (u8 0/1); per frame the mask count; per region of a
 *       4 x 4 grid (region of pixel (y, x) = (4y / H) * 4 + 4x / W, integer division) the
 *       mask pixels' count, sum of x and sum of y (int32 triples; frames whose sums
 *       could pass 2^31, max(W, H) (W H / 16 + W + H) >= 2^31, are rejected)
 *   K6  per region, a constant-velocity Kalman filter (state px, py, vx, vy; white
 *       acceleration q = 0.5 per frame; measurement = the region's mask centroid, noise
 *       r = 4 px^2; starts at the first frame with a measurement, P0 = diag(r, r, 100, 100))
 * Partitions of K1..K5: bit i of `cuts` (i = 0..3) cuts between K(i+1) and K(i+2); 0 is
 * "Full Fusion", 0b0010 (K1 K2 | K3 K4 K5) the paper's "Two Fusion", 0b1111 "No Fusion".
 * Maps between groups are FP32 planes of the workspace. Execution: 32 x 32 tiles of the
 * group's input (lanes = columns). The IIR recursion is cut into chunks of KF_PC_CHUNK
 * frames that run in parallel: the filter is linear, so a pass over the input gives each
 * chunk's end state from zero, a carry pass per pixel turns those into the true state
 * before every chunk (in chunk order), and a group holding K2 runs each (tile, chunk) as
 * one block of 8 warps from that state, 4 rows' states per warp in registers. The result
 * is the recursion evaluated in this fixed chunked order (the same in every partition);
 * other groups run one warp per (tile, frame). */
#define KF_PC_STAGES 5
#define KF_PC_CHUNK 32
#define KF_PC_REGIONS 16
typedef struct {
    const uint8_t *rgba;  /* device, T x H rows of `pitch` pixels of 4 bytes (R, G, B, A) */
    int64_t W, H, T;
    int64_t pitch;        /* pixels per row, >= W, a multiple of 4; rgba 16-byte aligned */
} kf_pc_video;
typedef struct {
    uint8_t *mask;        /* device, T x H x mask_pitch bytes, 16-byte aligned */
    int64_t mask_pitch;   /* >= W, a multiple of 4 */
    int32_t *counts;      /* device, [T], written (no pre-zeroing needed) */
    int32_t *regions;     /* device, [T][KF_PC_REGIONS][3] (count, sum x, sum y), written */
} kf_pc_out;
/* Predicted bytes moved by a partition (Sec. VI-D with the executor's 32 x 32 tiles: a
 * group reads its input tile with halo and writes its output tile; a group holding K2
 * also pays the chunked recursion: one more read of its input for the chunk end states,
 * the carry pass over one state plane per chunk, and the start states it reads, with
 * halo, per chunk -- the temporal halo of a box of KF_PC_CHUNK frames). */
kf_status kf_pc_traffic(kf_ctx *ctx, uint32_t cuts, int64_t W, int64_t H, int64_t T, double *bytes);
/* The partition of minimum predicted traffic (exact DP over the 16). */
kf_status kf_pc_plan(kf_ctx *ctx, int64_t W, int64_t H, int64_t T, uint32_t *cuts, double *bytes);
/* Workspace of a partition: the IIR chunk states (ceil(T / KF_PC_CHUNK) FP32 planes of
 * H x round_up(W, 8)), 32 partial copies of the per-frame sums (T x 32 x 49 int32), then
 * up to two FP32 maps of T x H x round_up(W, 8) between groups, each part 256-aligned. */
kf_status kf_pc_workspace_bytes(kf_ctx *ctx, uint32_t cuts, int64_t W, int64_t H, int64_t T, size_t *bytes);
/* Run K1..K5 in partition `cuts` on `stream` (asynchronous): one fused kernel per group
 * (plus the chunked recursion's two passes for the group holding K2), writing out->mask,
 * counts and regions. workspace: device, >= kf_pc_workspace_bytes, 256-byte aligned
 * (may be NULL when that is 0). */
kf_status kf_pc_run(kf_ctx *ctx, uint32_t cuts, const kf_pc_video *video, const kf_pc_out *out, void *workspace,
                    size_t workspace_bytes, void *stream);
/* One group [a..b] (0-based stages, a <= b <= 4) over explicit maps. in: a == 0 the RGBA
 * frames (video), else an FP32 map [T][H][in_pitch] of stage a-1. out: b == 4 the mask
 * outputs (out_mask), else an FP32 map [T][H][out_pitch] of stage b. Maps: 16-byte
 * aligned, pitches (elements) multiples of 4. A group holding K2
 * or ending at K5 needs a workspace of kf_pc_group_workspace_bytes (256-byte aligned):
 * the chunk states and the partial sums; other groups none. */
kf_status kf_pc_group_workspace_bytes(kf_ctx *ctx, int a, int b, int64_t W, int64_t H, int64_t T, size_t *bytes);
kf_status kf_pc_run_group(kf_ctx *ctx, int a, int b, const kf_pc_video *video, const float *in, int64_t in_pitch,
                          float *out, int64_t out_pitch, const kf_pc_out *out_mask, void *workspace,
                          size_t workspace_bytes, void *stream);
/* K6 over [T][n_tracks][3] region sums (device): states [T][n_tracks][4] (FP64, device) and
 * status [T][n_tracks] (0 not started, 1 updated, 2 predicted only). One thread per track
 * walks the frames in FP32; the x and y axes share one 2 x 2 covariance (the model is the
 * same per axis), which is the 4 x 4 filter's exact block structure. */
kf_status kf_pc_kalman(kf_ctx *ctx, const int32_t *regions, int64_t T, int n_tracks, double *states, int32_t *status,
                       void *stream);

/* ------------------------------------------------------------------ spatio-temporal boxes */
/* A fused group with a temporal reach, run over boxes of x * x pixels by t frames: the
 * input box of Alg. 2 (Sec. VI-C), the data utilisation of Eq. 3 and the box shape of
 * Eq. 5 / Eq. 6 (Sec. VI-E). The paper gives no stage with a finite temporal reach; the
 * group is the paper's chain with its IIR filter replaced by a finite one, over the same
 * RGBA input (kf_pc_video):
 *   K1  g = 77 R + 150 G + 29 B
 *   Kt  z_t = sum_{k=0..n} C(n, k) g_{max(t-n+k, 0)}, n in {1, 2, 4} (temporal reach n)
 *   K3  G = sum w(dy) w(dx) z(clamp(p + d)), w = [1 2 1]
 *   K4  M = |Sobel_x G| + |Sobel_y G|, indices clamped on G
 *   K5  mask = M > 261120 * 2^n (u8 0/1), i.e. M / (65280 * 2^n * 16) > 0.25; per frame
 *       the mask count
 * all in exact 32-bit integers. One-sided reaches dx = 2 (spatial, both sides), dt = n
 * (temporal, past side). */
/* Shared memory of one box: RGBA staging of one frame ((x + 8) x (x + 4) x 4 bytes), the
 * temporal map Kt of the same extent (4 bytes a pixel), the smoothed map (x + 2) x (x + 4)
 * x 4 bytes and the gray values of the n previous frames (2 bytes a pixel each). Box
 * sides x in {8, 16, 32, 48, 64, 96}; others are rejected. */
kf_status kf_st_smem_bytes(int n, int x, size_t *bytes);
/* Sec. VI-D's fused transfer for boxes x * x * t: model_bytes = B ((x + 4)^2 (t + n) * 4 +
 * x^2 t) with B = W H T / (x^2 t) (halos never clipped); clipped_bytes = the input
 * extents of the tiling's boxes clipped to the volume (4 bytes a pixel) + W H T mask
 * bytes. Either pointer may be NULL. */
kf_status kf_st_traffic(int64_t W, int64_t H, int64_t T, int x, int t, int n, double *model_bytes,
                        double *clipped_bytes);
/* Eq. 6 for this group's reaches (dx = 2, dt = n) and output volume beta = x^2 t:
 * x = (2 beta dx / dt)^(1/3), t = beta / x^2. */
kf_status kf_st_box_eq6(double beta, int n, double *x, double *t);
/* The supported box nearest Eq. 6 for output volume beta (>= 1): the side closest in
 * ratio to Eq. 6's x, t = beta / x^2 rounded (at least 1). */
kf_status kf_st_plan_eq6(double beta, int n, int *x, int *t);
/* The measured choice: runs kf_st_run once per candidate box (boxes[2 i], boxes[2 i + 1]
 * = x, t; one warm-up, `reps` timed runs, CUDA events on `stream`) and returns the
 * fastest box and its mean time. Every run writes mask and counts (the last one's stay).
 * Synchronous. */
kf_status kf_st_tune(kf_ctx *ctx, const kf_pc_video *video, uint8_t *mask, int64_t mask_pitch, int32_t *counts, int n,
                     const int *boxes, int count, int reps, void *stream, int *best_x, int *best_t, float *best_ms);
/* The group over the whole video in boxes of x * x * t (x as for kf_st_smem_bytes, t >=
 * 1), one block per box, frames streamed through shared memory in time order (the
 * temporal halo stays on chip for the box). mask: device, T x H x mask_pitch bytes (16-byte aligned,
 * mask_pitch >= W, a multiple of 4; the pitch padding is not written); counts: device
 * [T], written. A copy wait that runs out records KF_DEVERR_TIMEOUT. Asynchronous on
 * `stream`. */
kf_status kf_st_run(kf_ctx *ctx, const kf_pc_video *video, uint8_t *mask, int64_t mask_pitch, int32_t *counts, int n,
                    int x, int t, void *stream);

/* ------------------------------------------------------------------ kernel timing */
/* Per-kernel device time of the library's own launches (instrumentation; the paper
 * times whole kernels the same way, Sec. VI). While timing is on, kf_run, kf_run_group
 * and kf_track record a CUDA event pair on the launching stream around every kernel they
 * launch (the work itself is unchanged); kf_kernel_times waits for the recorded events
 * and returns, per kernel kind, the launches and their summed milliseconds since the
 * previous kf_kernel_times (or since timing was switched on), then clears the record.
 * Kinds: KF_KT_GROUP a fused group of the chain (kf_run, kf_run_group), KF_KT_CHAIN_CORNERS
 * the fully fused chain that also lists each frame's corners (kf_track), KF_KT_SELECT the
 * corner selection, KF_KT_LK the Lucas-Kanade step; kf_track_host also records its mask
 * packing kernels (KF_KT_PACK) and its copies (KF_KT_COPY_IN host to device,
 * KF_KT_COPY_OUT device to host), each on the stream that runs it. kf_set_kernel_timing
 * with on != 0 creates the events for 512 launches (more are created on demand beyond
 * that) and all are reused; KF_ECUDA if an event call fails. Not for use inside stream
 * capture. */
typedef enum {
    KF_KT_GROUP = 0,
    KF_KT_CHAIN_CORNERS = 1,
    KF_KT_SELECT = 2,
    KF_KT_LK = 3,
    KF_KT_PACK = 4,
    KF_KT_COPY_IN = 5,
    KF_KT_COPY_OUT = 6,
    KF_KT_COUNT = 7
} kf_kernel_kind;
kf_status kf_set_kernel_timing(kf_ctx *ctx, int on);
/* launches[KF_KT_COUNT], ms[KF_KT_COUNT]: host arrays */
kf_status kf_kernel_times(kf_ctx *ctx, int64_t *launches, double *ms);
/* The same record as a timeline: *n = the number of recorded launches and copies; the
 * first min(*n, cap) of them, in the order they were enqueued, go to kinds[i] (a
 * kf_kernel_kind), start_ms[i] and end_ms[i] (milliseconds from the earliest recorded
 * start, so that overlap between streams shows). Waits for the events and clears the
 * record, as kf_kernel_times does. KF_EINVAL if an array is null while cap > 0. */
kf_status kf_kernel_timeline(kf_ctx *ctx, int64_t cap, int64_t *n, int *kinds, double *start_ms, double *end_ms);

#ifdef __cplusplus
}
#endif
#endif /* KFUSE_H */
