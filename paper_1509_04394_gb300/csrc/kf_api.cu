// kf_api.cu -- host side of libkfuse.so: context, stage declarations, the partitioner
// (traffic model + exact dynamic program + enumeration) and the group executor.
//
// The partitioner is the model of Sec. VI (Fig. 5): choose contiguous groups covering
// every kernel exactly once so that the summed cost is minimal. With contiguous groups
// the constraint matrix has consecutive ones, so the 0/1 program is solved exactly by a
// shortest path over the n+1 cut points; the cost of a group is the traffic of Sec. VI-D
// (global<->on-chip bytes of one fused kernel) and a group is feasible when its on-chip
// footprint fits the limit (restriction c of Sec. VII).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/kfuse.h"
#include "kf_params.h"

#include "kf_ctx.h"
#include "kf_device.h"

namespace {

constexpr double NMS_THRESHOLD = 1e-5;  // on R in true units

bool builtin_chain(const kf_ctx *c)
{
    if ((int)c->stages.size() != kf::NSTAGES) return false;
    for (int i = 0; i < kf::NSTAGES; ++i)
        if (c->stages[i].kind != i + 1) return false;
    return true;
}

// bytes per pixel of the map written by 1-based stage k at a precision
double builtin_map_bytes(int k, int precision)
{
    if (k == 0 || k == 8) return 1.0;  // u8 frames, u8 mask
    return kf::map_channels(k) * (precision != KF_PREC_F32 ? 2.0 : 4.0);
}

kf_stage_desc builtin_desc(int kind, int precision)
{
    kf_stage_desc d{};
    d.kind = kind;
    d.rx = kf::stage_rx(kind);
    d.ry = kf::stage_ry(kind);
    d.rt = 0;
    d.in_bytes = builtin_map_bytes(kind - 1, precision);
    d.out_bytes = builtin_map_bytes(kind, precision);
    return d;
}

// effective descriptor: builtin kinds get their default byte counts where 0
kf_stage_desc eff(const kf_ctx *c, int i)
{
    kf_stage_desc d = c->stages[i];
    if (d.kind >= KF_STAGE_CONVERT && d.kind <= KF_STAGE_NMS) {
        const kf_stage_desc b = builtin_desc(d.kind, c->precision);
        if (d.in_bytes == 0) d.in_bytes = b.in_bytes;
        if (d.out_bytes == 0) d.out_bytes = b.out_bytes;
    }
    return d;
}

bool geom_ok(const kf_geometry *g) { return g && g->W > 0 && g->H > 0 && g->T > 0 && g->box_x >= 0 && g->box_y >= 0 && g->box_t >= 0; }

void box_of(const kf_ctx *c, const kf_geometry *g, double &x, double &y, double &t)
{
    x = g->box_x ? (double)g->box_x : (double)kf::strip_geometry(6, 1 << 20).step;
    y = g->box_y ? (double)g->box_y : (double)c->chunk_rows;
    t = g->box_t ? (double)g->box_t : 1.0;
}

void group_radii(const kf_ctx *c, int a, int b, double &rx, double &ry, double &rt)
{
    rx = ry = rt = 0;
    for (int k = a; k <= b; ++k) {
        rx += c->stages[k].rx;
        ry += c->stages[k].ry;
        rt += c->stages[k].rt;
    }
}

double traffic(const kf_ctx *c, int a, int b, const kf_geometry *g)
{
    double x, y, t, rx, ry, rt;
    box_of(c, g, x, y, t);
    group_radii(c, a, b, rx, ry, rt);
    const double boxes = (double)g->W * (double)g->H * (double)g->T / (x * y * t);
    const double per_box = (x + 2 * rx) * (y + 2 * ry) * (t + rt) * eff(c, a).in_bytes + x * y * t * eff(c, b).out_bytes;
    return boxes * per_box;
}

double onchip(const kf_ctx *c, int a, int b, const kf_geometry *g)
{
    double x, y, t, rx, ry, rt;
    box_of(c, g, x, y, t);
    group_radii(c, a, b, rx, ry, rt);
    double rows = 0;
    for (int k = a; k <= b; ++k) rows += (2.0 * c->stages[k].ry + 1.0) * eff(c, k).in_bytes;
    return (x + 2 * rx) * (t + rt) * rows;
}

kf_status cuda_fail(kf_ctx *c, cudaError_t e)
{
    c->last_cuda = (int)e;
    return KF_ECUDA;
}

kf::LaunchFn launcher(int A, int B, int f16)
{
    switch (A) {
    case 1: return kf::launcher_a1(B, f16);
    case 2: return kf::launcher_a2(B, f16);
    case 3: return kf::launcher_a3(B, f16);
    case 4: return kf::launcher_a4(B, f16);
    case 5: return kf::launcher_a5(B, f16);
    case 6: return kf::launcher_a6(B, f16);
    case 7: return kf::launcher_a7(B, f16);
    case 8: return kf::launcher_a8(B, f16);
    default: return nullptr;
    }
}

bool aligned(const void *p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
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

CUtensorMapDataType tmap_dtype(int dt)
{
    switch (dt) {
    case KF_DT_U8: return CU_TENSOR_MAP_DATA_TYPE_UINT8;
    case KF_DT_U16: return CU_TENSOR_MAP_DATA_TYPE_UINT16;
    case KF_DT_F16: return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    default: return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    }
}

int dtype_bytes(int dt) { return dt == KF_DT_U8 ? 1 : (dt == KF_DT_F32 ? 4 : 2); }

// 3-D descriptor {W, H, T} of one plane; box {box_x, RB, 1}; out-of-frame reads give 0.
bool encode_plane(CUtensorMap *m, const void *plane, int dt, int64_t pitch, int64_t fstride, int64_t W, int64_t H, int64_t T,
                  int box_x = kf::STRIP)
{
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const int e = dtype_bytes(dt);
    cuuint64_t dims[3] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)T};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * e), (cuuint64_t)(fstride * e)};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)kf::RB, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, tmap_dtype(dt), 3, const_cast<void *>(plane), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

int dtype_bytes(int dt);

// dtype of the map written by 1-based stage k (0 = frames)
int map_dtype(int k, int precision)
{
    if (k == 0 || k == 8) return KF_DT_U8;
    if (precision == KF_PREC_F32) return KF_DT_F32;
    return k <= 3 ? KF_DT_U16 : KF_DT_F16;
}

// map validation for kf_run_group: dtype/channels as the chain requires at this point
kf_status check_map(const kf_map *m, int stage_out, int precision, int64_t W, int64_t H)
{
    if (!m) return KF_EINVAL;
    const int want_dt = map_dtype(stage_out, precision);
    const int want_ch = kf::map_channels(stage_out);
    if (m->dtype != want_dt || m->channels != want_ch) return KF_EINVAL;
    const int64_t align_e = 16 / dtype_bytes(want_dt);  // rows and frames start on 16 bytes
    if (m->pitch < W || m->pitch % align_e || m->frame_stride < H * m->pitch || m->frame_stride % align_e) return KF_EINVAL;
    for (int i = 0; i < want_ch; ++i)
        if (!m->plane[i] || !aligned(m->plane[i], 16)) return KF_EINVAL;
    return KF_OK;
}

// Parameter block of group [A..B] (1-based) over already validated maps.
kf_status fill_params(kf_ctx *c, int A, int B, const kf_map &in, const kf_map &out, int64_t W, int64_t H, int64_t T,
                      int32_t *counts, unsigned long long *cand, int *cand_count, int64_t cand_cap, kf::GroupParams &p,
                      int chunk_rows = 0)
{
    const int rows = chunk_rows > 0 ? chunk_rows : c->chunk_rows;
    p = kf::GroupParams{};
    for (int i = 0; i < 3; ++i) {
        p.in[i] = in.plane[i];
        p.out[i] = out.plane[i];
    }
    for (int i = 0; i < in.channels; ++i)
        if (!encode_plane(&p.tmap[i], in.plane[i], in.dtype, in.pitch, in.frame_stride, W, H, T)) return KF_EINVAL;
    p.err = c->d_err;
    p.wait_polls = c->wait_polls;
    p.cand = cand;
    p.cand_count = cand_count;
    p.cand_cap = (int)cand_cap;
    p.in_pitch = in.pitch;
    p.in_fstride = in.frame_stride;
    p.out_pitch = out.pitch;
    p.out_fstride = out.frame_stride;
    p.counts = counts;
    p.W = (int)W;
    p.H = (int)H;
    const kf::StripGeom sg = kf::strip_geometry(kf::sum_rx(A, B), (int)W);
    p.xs0 = sg.xs0;
    p.step = sg.step;
    p.out_off = sg.out_off;
    p.n_strips = sg.n_strips;
    p.half_last = sg.half_last;
    p.n_lead = sg.n_lead;
    p.n_trail = sg.n_trail;
    if (p.half_last)
        for (int i = 0; i < in.channels; ++i)
            if (!encode_plane(&p.tmap_half[i], in.plane[i], in.dtype, in.pitch, in.frame_stride, W, H, T, kf::STRIP / 2))
                return KF_EINVAL;
    p.T = (int)T;
    p.chunk_rows = rows;
    p.n_chunks = (int)((H + rows - 1) / rows);
    p.n_jobs = T * p.n_chunks * (p.n_strips - p.half_last) + (T + 1) / 2 * p.n_chunks * p.half_last;
    p.thr = (float)(NMS_THRESHOLD * kf::map_scale(7));
    const bool f16 = c->precision != KF_PREC_F32;
    // FP16 maps (stages 4-7) hold true units; uint16 and FP32 maps hold scaled units
    p.in_scale = (f16 && A - 1 >= 4) ? (float)kf::map_scale(A - 1) : 1.0f;
    p.out_scale = (f16 && B >= 4 && B < 8) ? (float)(1.0 / kf::map_scale(B)) : 1.0f;
    if (p.n_jobs > 0x7fffffff) return KF_EINVAL;
    return KF_OK;
}

// Enqueue group [A..B] (1-based) with already validated maps.
// kernel timing: an event pair around one launch when the context's timing is on
cudaEvent_t timing_event(kf_ctx *c)
{
    if (!c->spare_events.empty()) {
        cudaEvent_t e = c->spare_events.back();
        c->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}
struct TimedLaunch {
    kf_ctx *c;
    int kind;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    TimedLaunch(kf_ctx *ctx, int k, cudaStream_t st) : c(ctx), kind(k), s(st)
    {
        if (!c->timing) return;
        a = timing_event(c);
        b = timing_event(c);
        if (a && b && cudaEventRecord(a, s) == cudaSuccess) return;
        if (a) c->spare_events.push_back(a);
        if (b) c->spare_events.push_back(b);
        a = b = nullptr;  // this launch goes untimed
    }
    void done()  // after a successful launch
    {
        if (!a) return;
        if (cudaEventRecord(b, s) == cudaSuccess) {
            c->timed.push_back({kind, a, b});
        } else {
            c->spare_events.push_back(a);
            c->spare_events.push_back(b);
        }
        a = b = nullptr;
    }
    ~TimedLaunch()
    {
        if (a) c->spare_events.push_back(a);
        if (b) c->spare_events.push_back(b);
    }
};

kf_status launch_group(kf_ctx *c, int A, int B, const kf_map &in, const kf_map &out, int64_t W, int64_t H, int64_t T,
                       int32_t *counts, cudaStream_t s, unsigned long long *cand = nullptr, int *cand_count = nullptr,
                       int64_t cand_cap = 0, int chunk_rows = 0, bool one_full_body = false,
                       unsigned long long *job_ctr = nullptr)
{
    if (T == 0) return KF_OK;
    kf::GroupParams p;
    kf_status st = fill_params(c, A, B, in, out, W, H, T, counts, cand, cand_count, cand_cap, p, chunk_rows);
    if (st != KF_OK) return st;
    p.one_full_body = one_full_body ? 1 : 0;
    if (job_ctr) {
        // jobs taken by SM: the share of SMs that start on interior strips follows the
        // interior strips' share of the work, a half-strip or edge job weighing 1.8
        // interior ones (measured best among 1.0-2.2 on the 1000 x 800 x 600 video: the
        // step 1.48 ms at 1.8 against 1.51 at 1.0 and 1.49 at 2.2, 267-row tiles)
        const int F = p.n_strips - p.half_last;
        const double n_other = (double)(p.n_jobs - (int64_t)T * p.n_chunks * F) +
                               (double)((int64_t)T * p.n_chunks * (p.n_lead + p.n_trail));
        const double n_in = (double)p.n_jobs - n_other;
        p.sm_split = n_in + n_other > 0 ? (int)(1024.0 * n_in / (n_in + 1.8 * n_other) + 0.5) : 1024;
        p.job_ctr = job_ctr;
        cudaError_t e = cudaMemsetAsync(job_ctr, 0, 3 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    // 0: FP32 maps; 1: 16-bit maps; 2: 16-bit maps and FP16 inter-stage tiles on chip
    const int f16 = c->precision == KF_PREC_F32 ? 0 : c->precision == KF_PREC_F16_TILES ? 2 : 1;
    const int64_t blocks = p.n_jobs;  // one warp (one job) per block
    if (B == 8) {
        cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * (size_t)T, s);
        if (e != cudaSuccess) return cuda_fail(c, e);
    }
    kf::LaunchFn fn = cand ? ((A == 1 && B == kf::NSTAGES) ? (f16 == 2 ? kf::launch_chain_with_candidates_tiles
                                                                      : kf::launch_chain_with_candidates)
                                                          : nullptr)
                           : launcher(A, B, f16);
    if (!fn) return KF_EINVAL;
    TimedLaunch tl(c, cand ? KF_KT_CHAIN_CORNERS : KF_KT_GROUP, s);
    const int e = fn(p, (unsigned)blocks, s);
    if (e != 0) return cuda_fail(c, (cudaError_t)e);
    tl.done();
    return KF_OK;
}

struct WsPlan {
    int64_t pitch_e = 0;      // elements per map row
    size_t plane_bytes = 0;   // one plane of the whole volume
    size_t buf_bytes[2] = {0, 0};
    size_t total = 0;
};

WsPlan plan_workspace(const kf_ctx *c, uint32_t cuts, int64_t W, int64_t H, int64_t T)
{
    WsPlan w;
    const size_t elem = c->precision != KF_PREC_F32 ? 2 : 4;
    w.pitch_e = round_up(W, 8);
    w.plane_bytes = (size_t)round_up((int64_t)(w.pitch_e * H * T * (int64_t)elem), 256);
    int k = 0;
    for (int i = 0; i < kf::NSTAGES - 1; ++i)
        if (cuts >> i & 1) {
            const size_t need = w.plane_bytes * (size_t)kf::map_channels(i + 1);
            if (need > w.buf_bytes[k % 2]) w.buf_bytes[k % 2] = need;
            ++k;
        }
    w.total = w.buf_bytes[0] + w.buf_bytes[1];
    return w;
}

}  // namespace

namespace kf {
int ctx_device(const kf_ctx *ctx) { return ctx ? ctx->device : -1; }
}  // namespace kf

extern "C" {

const char *kf_status_str(kf_status s)
{
    switch (s) {
    case KF_OK: return "ok";
    case KF_EINVAL: return "invalid argument";
    case KF_ENOMEM: return "out of memory or workspace too small";
    case KF_ECUDA: return "CUDA runtime error";
    case KF_ESMEM: return "group exceeds the on-chip limit";
    case KF_EUNSUPPORTED: return "chain cannot be executed";
    case KF_ESTATE: return "call not valid for this context";
    case KF_ETIMEOUT: return "device-side wait timed out";
    }
    return "unknown status";
}

int kf_last_cuda_error(const kf_ctx *ctx) { return ctx ? ctx->last_cuda : 0; }

kf_status kf_version(int *major, int *minor)
{
    if (!major || !minor) return KF_EINVAL;
    *major = KF_VERSION_MAJOR;
    *minor = KF_VERSION_MINOR;
    return KF_OK;
}

kf_status kf_create(int device, kf_ctx **out)
{
    if (!out) return KF_EINVAL;
    *out = nullptr;
    kf_ctx *c = new (std::nothrow) kf_ctx;
    if (!c) return KF_ENOMEM;
    c->device = device < 0 ? -1 : device;
    if (device >= 0) {
        kf::DeviceScope dev_scope(device);
    cudaError_t e = dev_scope.status();
        if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
        if (e != cudaSuccess) {
            if (c->d_err) cudaFree(c->d_err);
            delete c;
            return KF_ECUDA;
        }
    }
    *out = c;
    return KF_OK;
}

kf_status kf_destroy(kf_ctx *ctx)
{
    if (!ctx) return KF_OK;
    kf::costmodel_free(ctx);
    if (ctx->device >= 0) {  // device objects are released with their device current
        kf::DeviceScope dev_scope(ctx->device);
        if (ctx->s_in) {
            cudaStreamDestroy(ctx->s_in);
            cudaStreamDestroy(ctx->s_out);
            for (int i = 0; i < kf_ctx::N_RING; ++i) {
                cudaStreamDestroy(ctx->s_comp[i]);
                if (ctx->s_trk[i]) cudaStreamDestroy(ctx->s_trk[i]);
                cudaEventDestroy(ctx->ev_in[i]);
                cudaEventDestroy(ctx->ev_comp[i]);
                if (ctx->ev_chain[i]) cudaEventDestroy(ctx->ev_chain[i]);
            }
            cudaEventDestroy(ctx->ev_edge);
        }
        if (ctx->pack_buf) cudaFree(ctx->pack_buf);
        for (const kf_ctx::Timed &t : ctx->timed) {
            cudaEventDestroy(t.a);
            cudaEventDestroy(t.b);
        }
        for (cudaEvent_t e : ctx->spare_events) cudaEventDestroy(e);
        if (ctx->d_err) cudaFree(ctx->d_err);
    }
    delete ctx;
    return KF_OK;
}

kf_status kf_device_error(kf_ctx *ctx, int *code)
{
    if (!ctx || !code) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(code, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    return KF_OK;
}

kf_status kf_set_precision(kf_ctx *ctx, int precision)
{
    if (!ctx || (precision != KF_PREC_F32 && precision != KF_PREC_F16 && precision != KF_PREC_F16_TILES)) return KF_EINVAL;
    ctx->precision = precision;
    return KF_OK;
}

kf_status kf_set_chunk_rows(kf_ctx *ctx, int rows)
{
    if (!ctx || rows < 1) return KF_EINVAL;
    ctx->chunk_rows = rows;
    return KF_OK;
}

kf_status kf_set_host_chunk_rows(kf_ctx *ctx, int rows)
{
    if (!ctx || rows < 0) return KF_EINVAL;
    ctx->host_chunk_rows = rows;
    return KF_OK;
}

kf_status kf_set_wait_polls(kf_ctx *ctx, unsigned polls)
{
    if (!ctx) return KF_EINVAL;
    ctx->wait_polls = polls;
    return KF_OK;
}

kf_status kf_add_stage(kf_ctx *ctx, const kf_stage_desc *d, int *id)
{
    if (!ctx || !d) return KF_EINVAL;
    if ((int)ctx->stages.size() >= KF_MAX_STAGES) return KF_EINVAL;
    if (d->kind < KF_STAGE_CUSTOM || d->kind > KF_STAGE_NMS) return KF_EINVAL;
    if (d->rx < 0 || d->ry < 0 || d->rt < 0 || d->in_bytes < 0 || d->out_bytes < 0) return KF_EINVAL;
    if (d->kind == KF_STAGE_CUSTOM && (d->in_bytes <= 0 || d->out_bytes <= 0)) return KF_EINVAL;
    if (d->kind != KF_STAGE_CUSTOM && (d->rx != kf::stage_rx(d->kind) || d->ry != kf::stage_ry(d->kind) || d->rt != 0))
        return KF_EINVAL;  // builtin kinds have fixed radii
    ctx->stages.push_back(*d);
    if (id) *id = (int)ctx->stages.size() - 1;
    return KF_OK;
}

kf_status kf_add_harris_chain(kf_ctx *ctx)
{
    if (!ctx || !ctx->stages.empty()) return KF_EINVAL;
    for (int k = 1; k <= kf::NSTAGES; ++k) {
        kf_stage_desc d{};
        d.kind = k;
        d.rx = kf::stage_rx(k);
        d.ry = kf::stage_ry(k);
        ctx->stages.push_back(d);
    }
    return KF_OK;
}

kf_status kf_num_stages(const kf_ctx *ctx, int *n)
{
    if (!ctx || !n) return KF_EINVAL;
    *n = (int)ctx->stages.size();
    return KF_OK;
}

kf_status kf_group_traffic(const kf_ctx *ctx, int first, int last, const kf_geometry *g, double *bytes)
{
    if (!ctx || !bytes || !geom_ok(g)) return KF_EINVAL;
    if (first < 0 || last < first || last >= (int)ctx->stages.size()) return KF_EINVAL;
    *bytes = traffic(ctx, first, last, g);
    return KF_OK;
}

kf_status kf_group_onchip(const kf_ctx *ctx, int first, int last, const kf_geometry *g, double *bytes)
{
    if (!ctx || !bytes || !geom_ok(g)) return KF_EINVAL;
    if (first < 0 || last < first || last >= (int)ctx->stages.size()) return KF_EINVAL;
    *bytes = onchip(ctx, first, last, g);
    return KF_OK;
}

kf_status kf_partition_traffic(const kf_ctx *ctx, uint32_t cuts, const kf_geometry *g, double *bytes)
{
    if (!ctx || !bytes || !geom_ok(g)) return KF_EINVAL;
    const int n = (int)ctx->stages.size();
    if (n == 0 || (n - 1 < 32 && (cuts >> (n - 1)) != 0)) return KF_EINVAL;
    double tot = 0;
    int a = 0;
    for (int i = 0; i < n; ++i)
        if (i == n - 1 || (cuts >> i & 1)) {
            tot += traffic(ctx, a, i, g);
            a = i + 1;
        }
    *bytes = tot;
    return KF_OK;
}

kf_status kf_plan(const kf_ctx *ctx, const kf_geometry *g, double onchip_limit, uint32_t *cuts, double *bytes)
{
    if (!ctx || !cuts || !geom_ok(g) || !(onchip_limit > 0)) return KF_EINVAL;
    const int n = (int)ctx->stages.size();
    if (n == 0) return KF_EINVAL;
    // best[j]: cheapest cover of stages [0, j); from[j]: start of its last group
    std::vector<double> best(n + 1, INFINITY);
    std::vector<int> from(n + 1, -1);
    best[0] = 0;
    for (int j = 1; j <= n; ++j)
        for (int i = 0; i < j; ++i) {
            if (!std::isfinite(best[i])) continue;
            if (onchip(ctx, i, j - 1, g) > onchip_limit) continue;
            const double v = best[i] + traffic(ctx, i, j - 1, g);
            if (v < best[j]) {
                best[j] = v;
                from[j] = i;
            }
        }
    if (!std::isfinite(best[n])) return KF_ESMEM;
    uint32_t m = 0;
    for (int j = n; j > 0; j = from[j])
        if (from[j] > 0) m |= 1u << (from[j] - 1);
    *cuts = m;
    if (bytes) *bytes = best[n];
    return KF_OK;
}

kf_status kf_enumerate(const kf_ctx *ctx, uint32_t *buf, int64_t cap, int64_t *n_out)
{
    if (!ctx || !n_out || cap < 0 || (cap > 0 && !buf)) return KF_EINVAL;
    const int n = (int)ctx->stages.size();
    if (n == 0) return KF_EINVAL;
    const int64_t total = (int64_t)1 << (n - 1);
    for (int64_t i = 0; i < total && i < cap; ++i) buf[i] = (uint32_t)i;
    *n_out = total;
    return KF_OK;
}

kf_status kf_map_scale(const kf_ctx *ctx, int stage, double *factor)
{
    if (!ctx || !factor || stage < 0 || stage >= kf::NSTAGES) return KF_EINVAL;
    if (stage == kf::NSTAGES - 1 || (ctx->precision != KF_PREC_F32 && stage >= 3)) *factor = 1.0;
    else *factor = 1.0 / kf::map_scale(stage + 1);
    return KF_OK;
}

kf_status kf_workspace_bytes(const kf_ctx *ctx, uint32_t cuts, int64_t W, int64_t H, int64_t T, size_t *bytes)
{
    if (!ctx || !bytes || !kf::volume_ok(W, H, T)) return KF_EINVAL;
    if (cuts >> (kf::NSTAGES - 1)) return KF_EINVAL;
    *bytes = plan_workspace(ctx, cuts, W, H, T).total;
    return KF_OK;
}

kf_status kf_run_group(kf_ctx *ctx, int first, int last, const kf_map *in, const kf_map *out, int64_t W, int64_t H,
                       int64_t T, int32_t *counts, void *stream)
{
    if (!ctx) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    if (!builtin_chain(ctx)) return KF_EUNSUPPORTED;
    if (first < 0 || last < first || last >= kf::NSTAGES) return KF_EINVAL;
    if (W <= 0 || H <= 0 || T < 0 || W > (1 << 30) || H > (1 << 30)) return KF_EINVAL;
    const int A = first + 1, B = last + 1;
    kf_status s = check_map(in, A - 1, ctx->precision, W, H);
    if (s != KF_OK) return s;
    s = check_map(out, B, ctx->precision, W, H);
    if (s != KF_OK) return s;
    if (B == 8 && (!counts || !aligned(counts, 4))) return KF_EINVAL;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    return launch_group(ctx, A, B, *in, *out, W, H, T, counts, static_cast<cudaStream_t>(stream));
}

kf_status kf_run(kf_ctx *ctx, uint32_t cuts, const kf_video *v, const kf_corners *o, void *ws, size_t ws_bytes,
                 void *stream)
{
    if (!ctx) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    if (!builtin_chain(ctx)) return KF_EUNSUPPORTED;
    if (!v || !o) return KF_EINVAL;
    if (cuts >> (kf::NSTAGES - 1)) return KF_EINVAL;
    if (!kf::volume_ok(v->W, v->H, v->T)) return KF_EINVAL;
    if (v->pitch < v->W || v->pitch % 16 || o->mask_pitch < v->W || o->mask_pitch % 16) return KF_EINVAL;
    if (v->T == 0) return KF_OK;  // nothing to read or write
    if (!v->frames || !o->mask || !o->counts) return KF_EINVAL;
    if (!aligned(v->frames, 16) || !aligned(o->mask, 16) || !aligned(o->counts, 4)) return KF_EINVAL;
    const WsPlan w = plan_workspace(ctx, cuts, v->W, v->H, v->T);
    if (w.total > 0 && (!ws || !aligned(ws, 256))) return KF_EINVAL;
    if (ws_bytes < w.total) return KF_ENOMEM;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);

    kf_map cur{};
    cur.plane[0] = const_cast<uint8_t *>(v->frames);
    cur.channels = 1;
    cur.dtype = KF_DT_U8;
    cur.pitch = v->pitch;
    cur.frame_stride = v->pitch * v->H;
    int a = 1, k = 0;
    for (int b = 1; b <= kf::NSTAGES; ++b) {
        if (b < kf::NSTAGES && !(cuts >> (b - 1) & 1)) continue;
        kf_map nxt{};
        if (b == kf::NSTAGES) {
            nxt.plane[0] = o->mask;
            nxt.channels = 1;
            nxt.dtype = KF_DT_U8;
            nxt.pitch = o->mask_pitch;
            nxt.frame_stride = o->mask_pitch * v->H;
        } else {
            char *base = static_cast<char *>(ws) + (k % 2 ? w.buf_bytes[0] : 0);
            nxt.channels = kf::map_channels(b);
            for (int c = 0; c < nxt.channels; ++c) nxt.plane[c] = base + c * w.plane_bytes;
            nxt.dtype = map_dtype(b, ctx->precision);
            nxt.pitch = w.pitch_e;
            nxt.frame_stride = w.pitch_e * v->H;
            ++k;
        }
        kf_status st = launch_group(ctx, a, b, cur, nxt, v->W, v->H, v->T, o->counts, s);
        if (st != KF_OK) return st;
        cur = nxt;
        a = b + 1;
    }
    return KF_OK;
}

kf_status kf_track_workspace_bytes(const kf_ctx *ctx, int64_t W, int64_t H, int64_t T, size_t *bytes)
{
    if (!ctx || !bytes || !kf::volume_ok(W, H, T) || W * H > 0x7fffffffLL) return KF_EINVAL;
    // candidate counts, candidate lists, then three job counters for each chain launch
    // that may be in flight at once (one per compute stream of kf_track_host)
    static_assert(3 * 8 * kf_ctx::N_RING <= 256, "job counters");
    *bytes = (size_t)round_up(4 * T, 256) + (size_t)(8 * kf::cand_capacity(W, H) * T) + 256;
    return KF_OK;
}

namespace {

kf_status check_track_args(kf_ctx *ctx, const kf_video *v, const kf_corners *o, const kf_tracks *tr, void *ws,
                           size_t ws_bytes)
{
    if (!ctx) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    if (!builtin_chain(ctx)) return KF_EUNSUPPORTED;
    if (!v || !o || !tr) return KF_EINVAL;
    if (!kf::volume_ok(v->W, v->H, v->T) || v->W * v->H > 0x7fffffffLL) return KF_EINVAL;
    if (v->pitch < v->W || v->pitch % 16 || o->mask_pitch < v->W || o->mask_pitch % 16) return KF_EINVAL;
    if (tr->K < 1 || tr->K > 1024) return KF_EINVAL;
    if (v->T == 0) return KF_OK;
    if (!v->frames || !o->mask || !o->counts || !tr->n_points || !tr->idx || !tr->u || !tr->v || !tr->status)
        return KF_EINVAL;
    if (!aligned(v->frames, 16) || !aligned(o->mask, 16) || !aligned(o->counts, 4) || !aligned(tr->n_points, 4) ||
        !aligned(tr->idx, 4) || !aligned(tr->u, 4) || !aligned(tr->v, 4) || !aligned(tr->status, 4))
        return KF_EINVAL;
    size_t need = 0;
    if (kf_track_workspace_bytes(ctx, v->W, v->H, v->T, &need) != KF_OK) return KF_EINVAL;
    if (!ws || !aligned(ws, 256)) return KF_EINVAL;
    if (ws_bytes < need) return KF_ENOMEM;
    return KF_OK;
}

// The fusable set of the chain over frames [t0, t1): one fused kernel, which also lists
// each frame's corners in the workspace.
kf_status chain_range(kf_ctx *ctx, const kf_video *v, const kf_corners *o, void *ws, int64_t t0, int64_t t1,
                      cudaStream_t s, int chunk_rows = 0, bool one_full_body = false, int ctr_slot = -1)
{
    const int64_t n = t1 - t0;
    if (n <= 0) return KF_OK;
    int *cand_count = static_cast<int *>(ws);
    auto *cand = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + round_up(4 * v->T, 256));
    const int64_t cap = kf::cand_capacity(v->W, v->H);
    // jobs taken by SM kind with the counters of slot ctr_slot after the lists (launches
    // in flight at once use different slots; -1: jobs by block index)
    unsigned long long *job_ctr = ctr_slot >= 0 ? cand + cap * v->T + 3 * ctr_slot : nullptr;
    cudaError_t e = cudaMemsetAsync(cand_count + t0, 0, sizeof(int) * (size_t)n, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    const int64_t fstride = v->pitch * v->H, mstride = o->mask_pitch * v->H;
    kf_map fin{}, fout{};
    fin.plane[0] = const_cast<uint8_t *>(v->frames) + t0 * fstride;
    fin.channels = 1;
    fin.dtype = KF_DT_U8;
    fin.pitch = v->pitch;
    fin.frame_stride = fstride;
    fout.plane[0] = o->mask + t0 * mstride;
    fout.channels = 1;
    fout.dtype = KF_DT_U8;
    fout.pitch = o->mask_pitch;
    fout.frame_stride = mstride;
    return launch_group(ctx, 1, kf::NSTAGES, fin, fout, v->W, v->H, n, o->counts + t0, s, cand + t0 * cap,
                        cand_count + t0, cap, chunk_rows, one_full_body, job_ctr);
}

// The tracking set over frames [t0, t1), after the kernel-to-kernel dependency on the
// chain of those frames: selection, then LK (frame t0's LK reads frame t0 - 1).
kf_status tracking_range(kf_ctx *ctx, const kf_video *v, const kf_tracks *tr, void *ws, int64_t t0, int64_t t1,
                         cudaStream_t s)
{
    const int64_t n = t1 - t0;
    if (n <= 0) return KF_OK;
    kf::TrackVideo tv{};
    tv.frames = v->frames;
    tv.pitch = v->pitch;
    tv.W = (int)v->W;
    tv.H = (int)v->H;
    tv.T = (int)v->T;
    tv.cand = reinterpret_cast<unsigned long long *>(static_cast<char *>(ws) + round_up(4 * v->T, 256));
    tv.cand_count = static_cast<int *>(ws);
    tv.cand_cap = (int)kf::cand_capacity(v->W, v->H);
    tv.n_points = tr->n_points;
    tv.idx = tr->idx;
    tv.status = tr->status;
    tv.u = tr->u;
    tv.v = tr->v;
    tv.frame_begin = 0;
    tv.first_frame = t0;
    {
        TimedLaunch tl(ctx, KF_KT_SELECT, s);
        const int r = kf::launch_select(tv, nullptr, 1, n, tr->K, s);
        if (r) return cuda_fail(ctx, (cudaError_t)r);
        tl.done();
    }
    {
        TimedLaunch tl(ctx, KF_KT_LK, s);
        const int r = kf::launch_lk(tv, nullptr, 1, n, tr->K, s);
        if (r) return cuda_fail(ctx, (cudaError_t)r);
        tl.done();
    }
    return KF_OK;
}

// The hot path over frames [t0, t1) of a video whose frames [0, t1) are on the device:
// the chain with corner lists, then selection and LK, on s_trk after the chain's event
// when one is given.
kf_status track_range(kf_ctx *ctx, const kf_video *v, const kf_corners *o, const kf_tracks *tr, void *ws, int64_t t0,
                      int64_t t1, cudaStream_t s, cudaStream_t s_trk = nullptr, cudaEvent_t ev_chain = nullptr,
                      int chunk_rows = 0)
{
    kf_status st = chain_range(ctx, v, o, ws, t0, t1, s, chunk_rows, false, 0);
    if (st != KF_OK || t1 <= t0) return st;
    if (s_trk && ev_chain) {
        cudaError_t e = cudaEventRecord(ev_chain, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s_trk, ev_chain, 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
        s = s_trk;
    }
    return tracking_range(ctx, v, tr, ws, t0, t1, s);
}

// Bit-packing of the chain's masks for transfer: frame f's H * W pixels in raster order,
// pixel i as bit i % 8 of byte i / 8, 32 pixels (one 32-bit word) per thread, written to
// dst + f * dst_stride (a multiple of 16 bytes; the last word's bits past H * W are 0).
__global__ void __launch_bounds__(256) pack_mask_kernel(const uint8_t *__restrict__ mask, int64_t pitch, int64_t fstride,
                                                        int W, int H, int64_t n_frames, int64_t words, uint8_t *dst,
                                                        int64_t dst_stride)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= words) return;
    const int64_t p0 = i * 32, npx = (int64_t)W * H;
    const int y0 = (int)(p0 / W), x0 = (int)(p0 - (int64_t)y0 * W);
    const bool fast = x0 + 32 <= W && (x0 & 7) == 0 && (pitch & 7) == 0;
    for (int64_t f = blockIdx.y; f < n_frames; f += gridDim.y) {
        const uint8_t *fm = mask + f * fstride;
        uint32_t bits = 0;
        if (fast) {
            const uint2 *src = reinterpret_cast<const uint2 *>(fm + (int64_t)y0 * pitch + x0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint2 v = src[q];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t w = h ? v.y : v.x;  // 4 pixels; any nonzero byte is a set pixel
                    w |= w >> 4;
                    w |= w >> 2;
                    w |= w >> 1;
                    w &= 0x01010101u;
                    bits |= ((w | (w >> 7) | (w >> 14) | (w >> 21)) & 0xfu) << (8 * q + 4 * h);
                }
            }
        } else {
            int y = y0, xx = x0;
            for (int b = 0; b < 32 && p0 + b < npx; ++b) {
                bits |= (uint32_t)(fm[(int64_t)y * pitch + xx] != 0) << b;
                if (++xx == W) {
                    xx = 0;
                    ++y;
                }
            }
        }
        reinterpret_cast<uint32_t *>(dst + f * dst_stride)[i] = bits;
    }
}

// the context's copy streams and event ring (created on first use)
kf_status copy_streams(kf_ctx *c)
{
    if (c->s_in) return KF_OK;
    // the copy-out stream at the lowest priority: its mask-packing kernels fill SM slots
    // the chunks' chains leave free instead of taking them first (small blocks, many of
    // them); the tracking stream at the highest (it runs after every chain)
    int lo_prio = 0, hi_prio = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->s_out, cudaStreamNonBlocking, lo_prio);
    for (int i = 0; e == cudaSuccess && i < kf_ctx::N_RING; ++i) {
        e = cudaStreamCreateWithFlags(&c->s_comp[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->s_trk[i], cudaStreamNonBlocking, hi_prio);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_comp[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_chain[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_edge, cudaEventDisableTiming);
    return e == cudaSuccess ? KF_OK : cuda_fail(c, e);
}

}  // namespace

kf_status kf_track(kf_ctx *ctx, const kf_video *v, const kf_corners *o, const kf_tracks *tr, void *ws, size_t ws_bytes,
                   void *stream)
{
    kf_status st = check_track_args(ctx, v, o, tr, ws, ws_bytes);
    if (st != KF_OK || v->T == 0) return st;
    kf::DeviceScope dev_scope(ctx->device);
    const cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    return track_range(ctx, v, o, tr, ws, 0, v->T, static_cast<cudaStream_t>(stream));
}

kf_status kf_track_host(kf_ctx *ctx, const kf_video *host_video, const kf_corners *host_out,
                        const kf_tracks *host_tracks, const kf_video *video, const kf_corners *out,
                        const kf_tracks *tracks, void *workspace, size_t workspace_bytes, int64_t chunk, int mask_format,
                        void *stream)
{
    kf_status st = check_track_args(ctx, video, out, tracks, workspace, workspace_bytes);
    if (st != KF_OK) return st;
    if (!host_video || !host_out || !host_tracks || chunk < 1) return KF_EINVAL;
    if (mask_format != KF_MASK_BYTES && mask_format != KF_MASK_BITS) return KF_EINVAL;
    const int64_t T = video->T, H = video->H, K = tracks->K;
    const bool bits = mask_format == KF_MASK_BITS;
    const int64_t packed = (video->W * H + 7) / 8;
    if (host_video->W != video->W || host_video->H != H || host_video->T != T || host_video->pitch != video->pitch ||
        host_tracks->K != K)
        return KF_EINVAL;
    if (bits ? (host_out->mask_pitch < packed || host_out->mask_pitch % 16) : host_out->mask_pitch != out->mask_pitch)
        return KF_EINVAL;
    if (T == 0) return KF_OK;
    if (!host_video->frames || !host_out->mask || !host_out->counts || !host_tracks->n_points || !host_tracks->idx ||
        !host_tracks->u || !host_tracks->v || !host_tracks->status)
        return KF_EINVAL;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    // packed masks: staged per chunk in a device ring of N_RING chunks (owned by the
    // context, grown on demand) and copied out from there; a chunk holds at most
    // min(chunk, T) frames
    const int64_t slot_frames = chunk < T ? chunk : T;
    if (bits) {
        const size_t need = (size_t)kf_ctx::N_RING * (size_t)slot_frames * (size_t)host_out->mask_pitch;
        if (need > ctx->pack_bytes) {
            // the old ring may still be in use by an earlier call's copy-out stream
            e = ctx->s_out ? cudaStreamSynchronize(ctx->s_out) : cudaSuccess;
            if (e == cudaSuccess && ctx->pack_buf) e = cudaFree(ctx->pack_buf);
            ctx->pack_buf = nullptr;
            ctx->pack_bytes = 0;
            if (e == cudaSuccess) e = cudaMalloc(&ctx->pack_buf, need);
            if (e != cudaSuccess) {
                ctx->pack_buf = nullptr;
                return cuda_fail(ctx, e);
            }
            ctx->pack_bytes = need;
        }
    }
    if ((st = copy_streams(ctx)) != KF_OK) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the internal streams start after what the caller queued before this call
    e = cudaEventRecord(ctx->ev_edge, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_in, ctx->ev_edge, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_out, ctx->ev_edge, 0);
    for (int i = 0; e == cudaSuccess && i < kf_ctx::N_RING; ++i) e = cudaStreamWaitEvent(ctx->s_comp[i], ctx->ev_edge, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    const int64_t fstride = video->pitch * H, mstride = out->mask_pitch * H;
    // the first chunk is a quarter of the others, so the hot path starts sooner, and so is
    // the last one, so little of the hot path and of the copy out is left once the last
    // frames have arrived: after the first chunk, full chunks while more than a chunk and
    // a quarter remain, then the rest less a quarter chunk, then that quarter
    const int64_t first = chunk / 4 > 0 ? chunk / 4 : 1;
    // the tracking set runs in two launches of each kernel: over the frames up to the end
    // of the first chunk that reaches half of the video, once those chains are done (the
    // copies in still arriving), and over the rest after the last chain (measured on
    // 1000 x 800 x 600, 50-frame chunks: the call 2.76 ms against 2.80 with one tracking
    // launch after every chain, 2.77 with the first quarter, 2.85 with three quarters)
    const int64_t t_split = T / 2;
    int64_t split_at = 0;
    int64_t t1 = 0;
    for (int64_t t0 = 0, k = 0; t0 < T && e == cudaSuccess; t0 = t1, ++k) {
        const int64_t rest = T - t0;
        const int64_t len = k == 0 ? first : rest > chunk + first ? chunk : rest > first ? rest - first : rest;
        t1 = t0 + len < T ? t0 + len : T;
        const int64_t n = t1 - t0;
        const int r = (int)(k % kf_ctx::N_RING);
        cudaEvent_t ein = ctx->ev_in[r];
        const cudaStream_t cs = ctx->s_comp[r];
        // copy in (s_in), compute (the compute streams in turn), copy out (s_out). Chunks
        // touch disjoint frames of every buffer, and a chunk's tracking reads only input
        // frames copied in before it, so consecutive chunks' kernels may overlap: the next
        // chunks' launches fill the SMs while the previous one drains its last wave.
        {
            TimedLaunch tl(ctx, KF_KT_COPY_IN, ctx->s_in);
            e = cudaMemcpyAsync(const_cast<uint8_t *>(video->frames) + t0 * fstride, host_video->frames + t0 * fstride,
                                (size_t)(n * fstride), cudaMemcpyHostToDevice, ctx->s_in);
            if (e == cudaSuccess) tl.done();
        }
        if (e == cudaSuccess) e = cudaEventRecord(ein, ctx->s_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ein, 0);
        if (e != cudaSuccess) break;
        // chunk launches are about a wave long and run with other chunks' launches: one
        // full-strip loop body for all of them (measured: the call 2.82-2.92 ms against
        // 2.94-3.09 with interior strips on their own loop)
        st = chain_range(ctx, video, out, workspace, t0, t1, cs, ctx->host_chunk_rows, true, r);
        if (st != KF_OK) return st;
        // the masks leave after the chunk's chain
        e = cudaEventRecord(ctx->ev_chain[r], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_out, ctx->ev_chain[r], 0);
        auto d2h = [&](void *dst, const void *src, size_t bytes) {
            if (e != cudaSuccess) return;
            TimedLaunch tl(ctx, KF_KT_COPY_OUT, ctx->s_out);
            e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->s_out);
            if (e == cudaSuccess) tl.done();
        };
        if (bits) {
            // packed on the copy-out stream into ring slot r (the slot's previous chunk was
            // copied out earlier on the same stream), then copied out
            uint8_t *slot = ctx->pack_buf + (size_t)r * (size_t)slot_frames * (size_t)host_out->mask_pitch;
            const int64_t words = (packed + 3) / 4;
            const dim3 grid((unsigned)((words + 255) / 256), (unsigned)(n < 65535 ? n : 65535));
            if (e == cudaSuccess) {
                TimedLaunch tl(ctx, KF_KT_PACK, ctx->s_out);
                pack_mask_kernel<<<grid, 256, 0, ctx->s_out>>>(out->mask + t0 * mstride, out->mask_pitch, mstride,
                                                               (int)video->W, (int)H, n, words, slot,
                                                               host_out->mask_pitch);
                e = cudaGetLastError();
                if (e == cudaSuccess) tl.done();
            }
            // the packed words of each frame only; the rest of the host frame stride is untouched
            if (e == cudaSuccess) {
                TimedLaunch tl(ctx, KF_KT_COPY_OUT, ctx->s_out);
                e = cudaMemcpy2DAsync(host_out->mask + t0 * host_out->mask_pitch, (size_t)host_out->mask_pitch, slot,
                                      (size_t)host_out->mask_pitch, (size_t)(4 * words), (size_t)n, cudaMemcpyDeviceToHost,
                                      ctx->s_out);
                if (e == cudaSuccess) tl.done();
            }
        } else {
            d2h(host_out->mask + t0 * mstride, out->mask + t0 * mstride, (size_t)(n * mstride));
        }
        if (e == cudaSuccess && split_at == 0 && t_split > 0 && t1 >= t_split && t1 < T) {
            // every chunk up to this one: each compute stream's last chain event (earlier
            // chains on a stream come before it; a slot not recorded in this call holds an
            // earlier call's event, or none, and delays nothing of this call)
            const cudaStream_t ts = ctx->s_trk[0];
            for (int i = 0; e == cudaSuccess && i < kf_ctx::N_RING; ++i) e = cudaStreamWaitEvent(ts, ctx->ev_chain[i], 0);
            if (e != cudaSuccess) break;
            st = tracking_range(ctx, video, tracks, workspace, 0, t1, ts);
            if (st != KF_OK) return st;
            split_at = t1;
        }
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    // The tracking set of the frames from split_at on after every chunk's chain. Launched
    // per chunk, interleaved with the chunks' chains, the selection and LK blocks (up to
    // 106 KB of shared memory or 21 K registers each) wait for several chain blocks of an
    // SM to retire and keep its slots half empty meanwhile (measured: the call 3.1-3.4 ms
    // against 3.0 ms). Then the counts and tracks, one copy each.
    {
        const cudaStream_t ts = ctx->s_trk[0];
        for (int i = 0; e == cudaSuccess && i < kf_ctx::N_RING; ++i) e = cudaStreamWaitEvent(ts, ctx->ev_chain[i], 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e);
        st = tracking_range(ctx, video, tracks, workspace, split_at, T, ts);
        if (st != KF_OK) return st;
        e = cudaEventRecord(ctx->ev_comp[0], ts);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_out, ctx->ev_comp[0], 0);
    }
    auto d2h_all = [&](void *dst, const void *src, size_t bytes) {
        if (e != cudaSuccess) return;
        TimedLaunch tl(ctx, KF_KT_COPY_OUT, ctx->s_out);
        e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->s_out);
        if (e == cudaSuccess) tl.done();
    };
    d2h_all(host_out->counts, out->counts, sizeof(int32_t) * (size_t)T);
    d2h_all(host_tracks->n_points, tracks->n_points, sizeof(int32_t) * (size_t)T);
    d2h_all(host_tracks->idx, tracks->idx, sizeof(int32_t) * (size_t)(T * K));
    d2h_all(host_tracks->u, tracks->u, sizeof(float) * (size_t)(T * K));
    d2h_all(host_tracks->v, tracks->v, sizeof(float) * (size_t)(T * K));
    d2h_all(host_tracks->status, tracks->status, sizeof(int32_t) * (size_t)(T * K));
    // the caller's stream ends after the last copy out
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_edge, ctx->s_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->ev_edge, 0);
    return e == cudaSuccess ? KF_OK : cuda_fail(ctx, e);
}

kf_status kf_set_kernel_timing(kf_ctx *ctx, int on)
{
    if (!ctx) return KF_EINVAL;
    ctx->timing = on != 0;
    if (ctx->timing && ctx->device >= 0) {
        // the record's events are made here, not between the launches they time: creating
        // one may map memory for the device while kernels run
        kf::DeviceScope dev_scope(ctx->device);
        cudaError_t e = dev_scope.status();
        while (e == cudaSuccess && ctx->spare_events.size() < kf_ctx::TIMING_EVENTS) {
            cudaEvent_t ev = nullptr;
            e = cudaEventCreate(&ev);
            if (e == cudaSuccess) ctx->spare_events.push_back(ev);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e);
    }
    return KF_OK;
}

kf_status kf_kernel_timeline(kf_ctx *ctx, int64_t cap, int64_t *n, int *kinds, double *start_ms, double *end_ms)
{
    if (!ctx || !n || cap < 0 || (cap > 0 && (!kinds || !start_ms || !end_ms))) return KF_EINVAL;
    *n = (int64_t)ctx->timed.size();
    cudaError_t err = cudaSuccess;
    std::vector<double> t0, t1;
    if (!ctx->timed.empty()) {
        const cudaEvent_t ref = ctx->timed.front().a;
        for (const kf_ctx::Timed &t : ctx->timed) {
            float da = 0.f, db = 0.f;
            cudaError_t e = cudaEventSynchronize(t.b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&da, ref, t.a);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&db, ref, t.b);
            if (e != cudaSuccess && err == cudaSuccess) err = e;
            t0.push_back(da);
            t1.push_back(db);
        }
    }
    // times from the earliest start (a launch on another stream may start before the first
    // one recorded)
    double lo = 0.0;
    for (double v : t0) lo = v < lo ? v : lo;
    for (size_t i = 0; i < ctx->timed.size() && (int64_t)i < cap; ++i) {
        kinds[i] = ctx->timed[i].kind;
        start_ms[i] = t0[i] - lo;
        end_ms[i] = t1[i] - lo;
    }
    for (const kf_ctx::Timed &t : ctx->timed) {
        ctx->spare_events.push_back(t.a);
        ctx->spare_events.push_back(t.b);
    }
    ctx->timed.clear();
    return err == cudaSuccess ? KF_OK : cuda_fail(ctx, err);
}

kf_status kf_kernel_times(kf_ctx *ctx, int64_t *launches, double *ms)
{
    if (!ctx || !launches || !ms) return KF_EINVAL;
    for (int k = 0; k < KF_KT_COUNT; ++k) {
        launches[k] = 0;
        ms[k] = 0.0;
    }
    cudaError_t err = cudaSuccess;
    for (const kf_ctx::Timed &t : ctx->timed) {
        float dt = 0.f;
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&dt, t.a, t.b);
        if (e == cudaSuccess) {
            launches[t.kind] += 1;
            ms[t.kind] += dt;
        } else if (err == cudaSuccess) {
            err = e;
        }
        ctx->spare_events.push_back(t.a);
        ctx->spare_events.push_back(t.b);
    }
    ctx->timed.clear();
    return err == cudaSuccess ? KF_OK : cuda_fail(ctx, err);
}

}  // extern "C"

struct kf_batch {
    int device = -1;
    cudaGraphExec_t exec = nullptr;
};

namespace {

struct BatchLayout {
    size_t params = 0, items = 0, queue = 0, tracks = 0, cand_count = 0, cand = 0, total = 0;
};

BatchLayout batch_layout(const kf_video *videos, int n, bool track)
{
    BatchLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = (size_t)round_up((int64_t)(o + bytes), 256); return at; };
    L.params = take(sizeof(kf::GroupParams) * (size_t)n);
    L.items = take(sizeof(int64_t) * (size_t)(3 * n + 1));  // queue segments, kind-major
    L.queue = take(3 * sizeof(unsigned long long));  // one counter per kind of job
    if (track) {
        int64_t frames = 0, cand = 0;
        for (int i = 0; i < n; ++i) {
            frames += videos[i].T;
            cand += videos[i].T * kf::cand_capacity(videos[i].W, videos[i].H);
        }
        L.tracks = take(sizeof(kf::TrackVideo) * (size_t)n);
        L.cand_count = take(sizeof(int) * (size_t)frames);
        L.cand = take(sizeof(unsigned long long) * (size_t)cand);
    }
    L.total = o;
    return L;
}

bool video_ok(const kf_video *v)
{
    return v && v->T > 0 && kf::volume_ok(v->W, v->H, v->T) && v->W * v->H <= 0x7fffffffLL &&
           v->pitch >= v->W && v->pitch % 16 == 0 && v->frames && aligned(v->frames, 16);
}

}  // namespace

extern "C" {

kf_status kf_batch_workspace_bytes(const kf_ctx *ctx, const kf_video *videos, int n, int track_K, size_t *bytes)
{
    if (!ctx || !videos || n < 1 || !bytes || track_K < 0 || track_K > 1024) return KF_EINVAL;
    int64_t px = 0;  // the whole batch within the single-volume bound
    for (int i = 0; i < n; ++i) {
        const kf_video &v = videos[i];
        if (v.T <= 0 || !kf::volume_ok(v.W, v.H, v.T)) return KF_EINVAL;
        px += v.W * v.H * v.T;
        if (px > ((int64_t)1 << 46)) return KF_EINVAL;
    }
    *bytes = batch_layout(videos, n, track_K > 0).total;
    return KF_OK;
}

kf_status kf_batch_create(kf_ctx *ctx, const kf_video *videos, const kf_corners *outs, const kf_tracks *tracks, int n,
                          void *ws, size_t ws_bytes, kf_batch **out)
{
    return kf_batch_create_ex(ctx, videos, outs, tracks, n, nullptr, 0, ws, ws_bytes, out);
}

kf_status kf_batch_create_ex(kf_ctx *ctx, const kf_video *videos, const kf_corners *outs, const kf_tracks *tracks, int n,
                             const int *chunk_rows, int warps_per_sm, void *ws, size_t ws_bytes, kf_batch **out)
{
    if (!ctx || !videos || !outs || n < 1 || !out || warps_per_sm < 0) return KF_EINVAL;
    if (chunk_rows)
        for (int i = 0; i < n; ++i)
            if (chunk_rows[i] < 1) return KF_EINVAL;
    *out = nullptr;
    if (ctx->device < 0) return KF_ESTATE;
    if (!builtin_chain(ctx) || ctx->precision != KF_PREC_F32) return KF_EUNSUPPORTED;
    const bool track = tracks != nullptr;
    const int K = track ? tracks[0].K : 0;
    for (int i = 0; i < n; ++i) {
        const kf_video &v = videos[i];
        const kf_corners &o = outs[i];
        if (!video_ok(&v)) return KF_EINVAL;
        if (!o.mask || !o.counts || o.mask_pitch < v.W || o.mask_pitch % 16 || !aligned(o.mask, 16) || !aligned(o.counts, 4))
            return KF_EINVAL;
        if (track) {
            const kf_tracks &t = tracks[i];
            if (t.K != K || K < 1 || K > 1024 || !t.n_points || !t.idx || !t.u || !t.v || !t.status) return KF_EINVAL;
        }
    }
    const BatchLayout L = batch_layout(videos, n, track);
    if (!ws || !aligned(ws, 256)) return KF_EINVAL;
    if (ws_bytes < L.total) return KF_ENOMEM;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    char *base = static_cast<char *>(ws);
    auto *d_params = reinterpret_cast<kf::GroupParams *>(base + L.params);
    auto *d_items = reinterpret_cast<int64_t *>(base + L.items);
    auto *d_queue = reinterpret_cast<unsigned long long *>(base + L.queue);
    auto *d_tracks = reinterpret_cast<kf::TrackVideo *>(base + L.tracks);
    int *d_cand_count = reinterpret_cast<int *>(base + L.cand_count);
    auto *d_cand = reinterpret_cast<unsigned long long *>(base + L.cand);

    std::vector<kf::GroupParams> hp((size_t)n);
    std::vector<int64_t> items((size_t)(3 * n) + 1, 0);
    std::vector<kf::TrackVideo> ht(track ? (size_t)n : 0);
    int64_t frame_begin = 0, cand_off = 0;
    for (int i = 0; i < n; ++i) {
        const kf_video &v = videos[i];
        kf_map fin{}, fout{};
        fin.plane[0] = const_cast<uint8_t *>(v.frames);
        fin.channels = 1;
        fin.dtype = KF_DT_U8;
        fin.pitch = v.pitch;
        fin.frame_stride = v.pitch * v.H;
        fout.plane[0] = outs[i].mask;
        fout.channels = 1;
        fout.dtype = KF_DT_U8;
        fout.pitch = outs[i].mask_pitch;
        fout.frame_stride = outs[i].mask_pitch * v.H;
        const int64_t cap = track ? kf::cand_capacity(v.W, v.H) : 0;
        kf_status st = fill_params(ctx, 1, kf::NSTAGES, fin, fout, v.W, v.H, v.T, outs[i].counts,
                                   track ? d_cand + cand_off : nullptr, track ? d_cand_count + frame_begin : nullptr, cap,
                                   hp[(size_t)i], chunk_rows ? chunk_rows[i] : 0);
        if (st != KF_OK) return st;
        if (track) {
            kf::TrackVideo &tv = ht[(size_t)i];
            tv.frames = v.frames;
            tv.pitch = v.pitch;
            tv.W = (int)v.W;
            tv.H = (int)v.H;
            tv.T = (int)v.T;
            tv.cand = d_cand + cand_off;
            tv.cand_count = d_cand_count + frame_begin;
            tv.cand_cap = (int)cap;
            tv.n_points = tracks[i].n_points;
            tv.idx = tracks[i].idx;
            tv.status = tracks[i].status;
            tv.u = tracks[i].u;
            tv.v = tracks[i].v;
            tv.frame_begin = frame_begin;
        }
        frame_begin += v.T;
        cand_off += v.T * cap;
    }
    // The queue hands out the jobs of the videos in order of decreasing job length (rows
    // per job, then jobs per video), so the last jobs of the launch are the shortest and
    // the tail of the persistent launch is short (longest-job-first order).
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const kf::GroupParams &pa = hp[(size_t)a], &pb = hp[(size_t)b];
        if (pa.chunk_rows != pb.chunk_rows) return pa.chunk_rows > pb.chunk_rows;
        return pa.n_jobs > pb.n_jobs;
    });
    std::vector<kf::GroupParams> hq((size_t)n);
    for (int k = 0; k < n; ++k) hq[(size_t)k] = hp[(size_t)order[(size_t)k]];
    // queue segments, kind-major (the batch kernel's order): half-strip jobs of every
    // video, then edge-strip jobs, then interior-strip jobs, each in the longest-first order
    for (int kind = 0, s = 0; kind < 3; ++kind)
        for (int k = 0; k < n; ++k, ++s) {
            const kf::GroupParams &q = hq[(size_t)k];
            const int F = q.n_strips - q.half_last;
            const int64_t per = (int64_t)q.T * q.n_chunks;
            const int64_t cnt = kind == 0 ? q.n_jobs - per * F
                              : kind == 1 ? per * (q.n_lead + q.n_trail)
                                          : per * (F - q.n_lead - q.n_trail);
            items[(size_t)s + 1] = items[(size_t)s] + cnt;
        }
    e = cudaMemcpy(d_params, hq.data(), sizeof(kf::GroupParams) * (size_t)n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_items, items.data(), sizeof(int64_t) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && track)
        e = cudaMemcpy(d_tracks, ht.data(), sizeof(kf::TrackVideo) * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e);

    // one CUDA graph: reset the queue and counters, the persistent chain, selection, LK
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    int per_sm = kf::batch_chain_blocks_per_sm(track);
    if (per_sm < 1) return cuda_fail(ctx, cudaErrorInvalidConfiguration);
    if (warps_per_sm > 0 && warps_per_sm < per_sm) per_sm = warps_per_sm;  // one warp per block
    if (track) {
        const int r = kf::prepare_select();
        if (r) return cuda_fail(ctx, (cudaError_t)r);
    }
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_queue, 0, 3 * sizeof(unsigned long long), cs);
    if (e == cudaSuccess && track) e = cudaMemsetAsync(d_cand_count, 0, sizeof(int) * (size_t)frame_begin, cs);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaMemsetAsync(outs[i].counts, 0, sizeof(int32_t) * (size_t)videos[i].T, cs);
    if (e == cudaSuccess) {
        // the share of SMs that start on interior strips, as in a single video's launch
        const double n_in = (double)(items[(size_t)(3 * n)] - items[(size_t)(2 * n)]);
        const double n_other = (double)items[(size_t)(2 * n)];
        const int sm_split = n_in + n_other > 0 ? (int)(1024.0 * n_in / (n_in + 1.8 * n_other) + 0.5) : 1024;
        const int r = kf::launch_batch_chain(d_params, d_items, n, d_queue, track, (unsigned)(sms * per_sm), sm_split, cs);
        if (r) e = (cudaError_t)r;
    }
    if (e == cudaSuccess && track) {
        const kf::TrackVideo none{};
        int r = kf::launch_select(none, d_tracks, n, frame_begin, K, cs);
        if (!r) r = kf::launch_lk(none, d_tracks, n, frame_begin, K, cs);
        if (r) e = (cudaError_t)r;
    }
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    kf_batch *b = new (std::nothrow) kf_batch;
    if (!b) {
        cudaGraphExecDestroy(exec);
        return KF_ENOMEM;
    }
    b->device = ctx->device;
    b->exec = exec;
    *out = b;
    return KF_OK;
}

kf_status kf_batch_run(kf_batch *b, void *stream)
{
    if (!b || !b->exec) return KF_EINVAL;
    kf::DeviceScope dev_scope(b->device);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
    return cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? KF_OK : KF_ECUDA;
}

kf_status kf_batch_destroy(kf_batch *b)
{
    if (b) {
        kf::DeviceScope dev_scope(b->device);
        if (b->exec) {
            cudaGraphExecDestroy(b->exec);
        }
        delete b;
    }
    return KF_OK;
}

kf_status kf_tune_chunk_rows(kf_ctx *ctx, const kf_video *v, const kf_corners *o, const int *candidates, int n, int reps,
                             void *stream, int *best_rows, float *best_ms)
{
    if (!ctx || !v || !o || !candidates || n < 1 || reps < 1 || !best_rows) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    for (int i = 0; i < n; ++i)
        if (candidates[i] < 1) return KF_EINVAL;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return KF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KF_ECUDA;
    }
    const int keep = ctx->chunk_rows;
    int best = keep;
    float best_t = INFINITY;
    kf_status st = KF_OK;
    for (int i = 0; i < n && st == KF_OK; ++i) {
        ctx->chunk_rows = candidates[i];
        st = kf_run(ctx, 0, v, o, nullptr, 0, stream);  // warm-up
        if (st != KF_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == KF_OK; ++r) st = kf_run(ctx, 0, v, o, nullptr, 0, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = KF_ECUDA;
        float ms = 0;
        if (st == KF_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / reps < best_t) {
            best_t = ms / reps;
            best = candidates[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->chunk_rows = st == KF_OK ? best : keep;
    if (st != KF_OK) return st;
    *best_rows = best;
    if (best_ms) *best_ms = best_t;
    return KF_OK;
}

kf_status kf_tune_track_rows(kf_ctx *ctx, const kf_video *v, const kf_corners *o, const kf_tracks *tr, void *ws,
                             size_t ws_bytes, const int *candidates, int n, int reps, void *stream, int *best_rows,
                             float *best_ms)
{
    if (!ctx || !v || !o || !tr || !candidates || n < 1 || reps < 1 || !best_rows) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    for (int i = 0; i < n; ++i)
        if (candidates[i] < 1) return KF_EINVAL;
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return KF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KF_ECUDA;
    }
    const int keep = ctx->chunk_rows;
    int best = keep;
    float best_t = INFINITY;
    kf_status st = KF_OK;
    for (int i = 0; i < n && st == KF_OK; ++i) {
        ctx->chunk_rows = candidates[i];
        st = kf_track(ctx, v, o, tr, ws, ws_bytes, stream);  // warm-up
        if (st != KF_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == KF_OK; ++r) st = kf_track(ctx, v, o, tr, ws, ws_bytes, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = KF_ECUDA;
        float ms = 0;
        if (st == KF_OK && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms / reps < best_t) {
            best_t = ms / reps;
            best = candidates[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->chunk_rows = st == KF_OK ? best : keep;
    if (st != KF_OK) return st;
    *best_rows = best;
    if (best_ms) *best_ms = best_t;
    return KF_OK;
}

kf_status kf_plan_measured(kf_ctx *ctx, const kf_video *v, const kf_corners *o, void *ws, size_t ws_bytes,
                           const uint32_t *cands, int n_cand, int reps, void *stream, uint32_t *best_cuts, float *best_ms,
                           float *ms_all)
{
    if (!ctx || !v || !o || reps < 1 || !best_cuts || (cands && n_cand < 1)) return KF_EINVAL;
    if (ctx->device < 0) return KF_ESTATE;
    if (!builtin_chain(ctx)) return KF_EUNSUPPORTED;
    const int n_all = 1 << (kf::NSTAGES - 1);
    const int n = cands ? n_cand : n_all;
    for (int i = 0; i < n; ++i) {
        const uint32_t c = cands ? cands[i] : (uint32_t)i;
        if (c >= (uint32_t)n_all) return KF_EINVAL;
        if (plan_workspace(ctx, c, v->W, v->H, v->T).total > ws_bytes) return KF_ENOMEM;
    }
    kf::DeviceScope dev_scope(ctx->device);
    cudaError_t e = dev_scope.status();
    if (e != cudaSuccess) return cuda_fail(ctx, e);
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::vector<cudaEvent_t> ev(2 * (size_t)reps, nullptr);
    kf_status st = KF_OK;
    for (cudaEvent_t &x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) st = KF_ECUDA;
    uint32_t best = 0;
    float best_t = INFINITY;
    std::vector<float> t((size_t)reps);
    for (int i = 0; i < n && st == KF_OK; ++i) {
        const uint32_t c = cands ? cands[i] : (uint32_t)i;
        st = kf_run(ctx, c, v, o, ws, ws_bytes, stream);  // warm-up
        for (int r = 0; r < reps && st == KF_OK; ++r) {
            cudaEventRecord(ev[2 * r], s);
            st = kf_run(ctx, c, v, o, ws, ws_bytes, stream);
            cudaEventRecord(ev[2 * r + 1], s);
        }
        if (st == KF_OK && cudaEventSynchronize(ev[2 * reps - 1]) != cudaSuccess) st = KF_ECUDA;
        for (int r = 0; r < reps && st == KF_OK; ++r)
            if (cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]) != cudaSuccess) st = KF_ECUDA;
        if (st != KF_OK) break;
        std::sort(t.begin(), t.end());
        const float med = t[(size_t)reps / 2];  // median (upper median for even counts)
        if (ms_all) ms_all[i] = med;
        if (med < best_t) {
            best_t = med;
            best = c;
        }
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (st != KF_OK) return st;
    *best_cuts = best;
    if (best_ms) *best_ms = best_t;
    return KF_OK;
}

}  // extern "C"
