// kf_dag.cu -- fused execution of arbitrary kernel DAGs (the learned cost model's workload).
//
// A DAG of generic stages (affine, abs, saturating product, separable binomial stencil
// of radius 0..3, 3x3 maximum; one or two inputs each, node 0 = the frame as u8/255) is
// cut into contiguous groups of its topological order, and each group runs as one fused
// kernel written the way Alg. 1 states it: every block copies its input box (the tile
// plus the group's halo, per external input) from global to shared memory, runs the
// group's stages one after the other on shared-memory tiles with a barrier between
// stages (every stage here is thread-to-multi-thread, Sec. V-A b), and stores only the
// maps later groups read. Each node is computed over the tile grown by its own halo, the
// largest (consumer halo + consumer radius) over its consumers in the group (Alg. 2 with
// radii summed along paths). Every stencil clamps its own input: a node's value outside
// the frame is its value at the clamped position, so each region position computes the
// stage at the clamped position. Shared-memory slots are reused once a node's last
// consumer in the group has run; a group whose slots exceed the on-chip limit is
// infeasible (restriction c of Sec. VII).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/kfuse.h"
#include "kf_ctx.h"
#include "kf_device.h"

namespace kf {
int ctx_device(const kf_ctx *ctx);
// the learned model's prediction of one group on the host (kf_mlp.cu)
kf_status predict_group_ms(kf_ctx *model, const float *features, float *ms);
}

namespace {

constexpr int DAG_TX = 32, DAG_TY = 16;  // output tile of a block
constexpr int DAG_THREADS = 256;
constexpr int DAG_MAX_OPS = 2 * KF_DAG_MAX_STAGES;
constexpr double DAG_SMEM_LIMIT = 200.0 * 1024;  // bytes of shared memory a block may use

struct DagOp {
    int kind;  // 0 = load node `node` (frame or map), else KF_G_* of stage `node`
    int node;
    int out_slot, in1_slot, in2_slot;
    int halo, in1_halo, in2_halo;
    int radius;
    float a, b;
    int store;  // 1: write the tile interior to the node's map
};

struct DagProg {
    int n_ops;
    int slot_floats;
    DagOp ops[DAG_MAX_OPS];
};

__constant__ float c_binom[4][7] = {
    {1.0f, 0, 0, 0, 0, 0, 0},
    {0.25f, 0.5f, 0.25f, 0, 0, 0, 0},
    {1.0f / 16, 4.0f / 16, 6.0f / 16, 4.0f / 16, 1.0f / 16, 0, 0},
    {1.0f / 64, 6.0f / 64, 15.0f / 64, 20.0f / 64, 15.0f / 64, 6.0f / 64, 1.0f / 64},
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// maps: node j's map at maps + j * plane (floats, row pitch `pitch`); node `out_node`
// goes to `out` instead.
__global__ void __launch_bounds__(DAG_THREADS) dag_group_kernel(const __grid_constant__ DagProg prog,
                                                               const uint8_t *frames, int64_t fpitch, float *maps,
                                                               int64_t plane, int64_t pitch, float *out, int64_t opitch,
                                                               int out_node, int W, int H)
{
    extern __shared__ float sm[];
    const int x0 = blockIdx.x * DAG_TX, y0 = blockIdx.y * DAG_TY;
    const int64_t frame = blockIdx.z;
    for (int k = 0; k < prog.n_ops; ++k) {
        const DagOp &op = prog.ops[k];
        const int h = op.halo, RW = DAG_TX + 2 * h, RH = DAG_TY + 2 * h;
        float *dst = sm + (int64_t)op.out_slot * prog.slot_floats;
        const float *s1 = sm + (int64_t)op.in1_slot * prog.slot_floats;
        const float *s2 = sm + (int64_t)op.in2_slot * prog.slot_floats;
        const int R1 = DAG_TX + 2 * op.in1_halo, R2 = DAG_TX + 2 * op.in2_halo;
        // origin of the input regions in frame coordinates
        const int oy1 = y0 - op.in1_halo, ox1 = x0 - op.in1_halo, oy2 = y0 - op.in2_halo, ox2 = x0 - op.in2_halo;
        float *map_out = op.node == out_node ? out + frame * H * opitch : maps + op.node * plane + frame * H * pitch;
        const int64_t mp = op.node == out_node ? opitch : pitch;
        for (int i = threadIdx.x; i < RW * RH; i += DAG_THREADS) {
            const int py = i / RW, px = i - py * RW;
            const int gy = y0 - h + py, gx = x0 - h + px;
            const int qy = clampi(gy, 0, H - 1), qx = clampi(gx, 0, W - 1);
            float v;
            if (op.kind == 0) {
                if (op.node == 0) v = (float)frames[frame * H * fpitch + (int64_t)qy * fpitch + qx] * (1.0f / 255.0f);
                else v = maps[op.node * plane + frame * H * pitch + (int64_t)qy * pitch + qx];
            } else {
                const int ly = qy - oy1, lx = qx - ox1;  // the clamped position in input 1's region
                switch (op.kind) {
                case KF_G_AFFINE: v = fmaf(op.a, s1[ly * R1 + lx], op.b); break;
                case KF_G_ABS: v = fabsf(s1[ly * R1 + lx]); break;
                case KF_G_PRODUCT: {
                    const float p = s1[ly * R1 + lx] * s2[(qy - oy2) * R2 + (qx - ox2)];
                    v = fminf(fmaxf(p, -16.0f), 16.0f);
                    break;
                }
                case KF_G_STENCIL: {
                    const int r = op.radius;
                    v = 0.0f;
                    for (int dy = -r; dy <= r; ++dy) {
                        float row = 0.0f;
                        for (int dx = -r; dx <= r; ++dx) row = fmaf(c_binom[r][dx + r], s1[(ly + dy) * R1 + lx + dx], row);
                        v = fmaf(c_binom[r][dy + r], row, v);
                    }
                    break;
                }
                default: {  // KF_G_MAX3
                    v = s1[ly * R1 + lx];
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) v = fmaxf(v, s1[(ly + dy) * R1 + lx + dx]);
                    break;
                }
                }
            }
            dst[i] = v;
            if (op.store && py >= h && py < h + DAG_TY && px >= h && px < h + DAG_TX && gy < H && gx < W)
                map_out[(int64_t)gy * mp + gx] = v;
        }
        __syncthreads();
    }
}

}  // namespace

struct kf_dag {
    int device = -1;
    int n = 0;
    std::vector<kf_gstage> st;           // st[i-1] writes node i
    std::vector<std::vector<int>> cons;  // consumers (stage indices) of node j
};

namespace {

struct GroupPlan {
    bool feasible = false;
    DagProg prog{};
    double smem_bytes = 0;
    std::vector<int> ext;     // external input nodes
    std::vector<int> ext_h;   // their halos
    std::vector<int> outs;    // nodes stored
    std::vector<int> halo;    // halo per node (index node), -1 if not computed
    int peak_slots = 0;
};

int stage_radius(const kf_gstage &s) { return s.kind == KF_G_STENCIL ? s.radius : (s.kind == KF_G_MAX3 ? 1 : 0); }

// Node masks: bit j-1 stands for node j (1..n).
inline bool has(uint32_t m, int j) { return j >= 1 && (m >> (j - 1) & 1u); }
uint32_t range_mask(int a, int b) { return (b >= 32 ? ~0u : ((1u << b) - 1u)) & ~((1u << (a - 1)) - 1u); }

// The group of range [a, b] when the nodes of X are inlined (recomputed by every group
// that needs them instead of being stored): the range's nodes that are not inlined or
// are needed by a range node, plus, transitively, the inlined inputs of its members.
uint32_t members_of(const kf_dag *d, int a, int b, uint32_t X)
{
    uint32_t m = 0;
    for (int j = b; j >= a; --j) {
        bool need = !has(X, j);
        for (int c : d->cons[j]) need = need || has(m, c);
        if (need) m |= 1u << (j - 1);
    }
    for (int j = b; j >= 1; --j) {  // inputs are lower-numbered: one descending sweep closes the set
        if (!has(m, j)) continue;
        const kf_gstage &s = d->st[j - 1];
        for (int in : {s.in1, s.kind == KF_G_PRODUCT ? s.in2 : 0})
            if (in >= 1 && has(X, in)) m |= 1u << (in - 1);
    }
    return m;
}

// The range nodes the group stores: the output, and every node not inlined from which a
// path through inlined nodes reaches a stage after the range.
uint32_t stores_of(const kf_dag *d, int a, int b, uint32_t X)
{
    const int n = d->n;
    // reach[j]: the highest stage reachable from j through inlined intermediates
    std::vector<int> reach(n + 1, 0);
    for (int j = n; j >= 1; --j) {
        int r = 0;
        for (int c : d->cons[j]) r = std::max(r, has(X, c) ? std::max(c, reach[c]) : c);
        reach[j] = r;
    }
    uint32_t m = 0;
    for (int j = a; j <= b; ++j)
        if (j == n || (!has(X, j) && reach[j] > b)) m |= 1u << (j - 1);
    return m;
}

// program of a group computing the nodes of `members` and storing those of `outs`
GroupPlan plan_members(const kf_dag *d, uint32_t members, uint32_t outs)
{
    GroupPlan g;
    const int n = d->n;
    g.halo.assign(n + 1, -1);
    int top = 0;
    for (int j = n; j >= 1; --j)
        if (has(members, j)) {
            top = j;
            break;
        }
    for (int j = top; j >= 1; --j) {
        if (!has(members, j)) continue;
        int h = has(outs, j) ? 0 : -1;
        for (int c : d->cons[j])
            if (has(members, c) && g.halo[c] >= 0) h = std::max(h, g.halo[c] + stage_radius(d->st[c - 1]));
        g.halo[j] = h;
        if (has(outs, j)) g.outs.push_back(j);
    }
    for (int e = 0; e < top; ++e) {
        if (has(members, e)) continue;
        int h = -1;
        for (int c : d->cons[e])
            if (has(members, c) && g.halo[c] >= 0) h = std::max(h, g.halo[c] + stage_radius(d->st[c - 1]));
        if (h >= 0) {
            g.ext.push_back(e);
            g.ext_h.push_back(h);
            g.halo[e] = h;
        }
    }
    // last consumer in the group of every live node
    std::vector<int> last(n + 1, -1);
    for (int j = 0; j <= top; ++j)
        for (int c : d->cons[j])
            if (has(members, c) && g.halo[c] >= 0) last[j] = std::max(last[j], c);
    int hmax = 0;
    for (int j = 0; j <= top; ++j) hmax = std::max(hmax, g.halo[j]);
    const int slot_floats = (DAG_TX + 2 * hmax) * (DAG_TY + 2 * hmax);
    std::vector<int> slot_of(n + 1, -1);
    std::vector<int> free_slots;
    int n_slots = 0;
    auto take = [&]() {
        if (!free_slots.empty()) {
            const int s = free_slots.back();
            free_slots.pop_back();
            return s;
        }
        return n_slots++;
    };
    int nops = 0;
    for (size_t i = 0; i < g.ext.size(); ++i) {
        DagOp &op = g.prog.ops[nops++];
        op = DagOp{};
        op.kind = 0;
        op.node = g.ext[i];
        op.halo = g.ext_h[i];
        op.out_slot = slot_of[op.node] = take();
    }
    for (int j = 1; j <= top; ++j) {
        if (!has(members, j) || g.halo[j] < 0) continue;  // not a member, or nothing stored depends on it
        const kf_gstage &s = d->st[j - 1];
        DagOp &op = g.prog.ops[nops++];
        op = DagOp{};
        op.kind = s.kind;
        op.node = j;
        op.halo = g.halo[j];
        op.radius = s.radius;
        op.a = s.a;
        op.b = s.b;
        op.in1_slot = slot_of[s.in1];
        op.in1_halo = g.halo[s.in1];
        op.in2_slot = s.kind == KF_G_PRODUCT ? slot_of[s.in2] : 0;
        op.in2_halo = s.kind == KF_G_PRODUCT ? g.halo[s.in2] : 0;
        op.store = has(outs, j) ? 1 : 0;
        op.out_slot = slot_of[j] = take();
        // free the inputs whose last in-group consumer is this stage (after writing j's slot)
        for (int in : {s.in1, s.kind == KF_G_PRODUCT ? s.in2 : -1})
            if (in >= 0 && last[in] == j && slot_of[in] >= 0) {
                free_slots.push_back(slot_of[in]);
                slot_of[in] = -1;
            }
        g.peak_slots = std::max(g.peak_slots, n_slots);
    }
    g.peak_slots = std::max(g.peak_slots, n_slots);
    g.prog.n_ops = nops;
    g.prog.slot_floats = slot_floats;
    g.smem_bytes = (double)n_slots * slot_floats * sizeof(float);
    g.feasible = g.smem_bytes <= DAG_SMEM_LIMIT;
    return g;
}

// group of nodes [a, b] (1-based, inclusive) of a contiguous partition
GroupPlan plan_group(const kf_dag *d, int a, int b) { return plan_members(d, range_mask(a, b), stores_of(d, a, b, 0)); }

// Sec. VI-D over the executor's tile: halo'd input boxes in, stored maps out (bytes per tile)
double tile_traffic(const GroupPlan &g)
{
    double per_box = 0;
    for (size_t i = 0; i < g.ext.size(); ++i)
        per_box += (DAG_TX + 2.0 * g.ext_h[i]) * (DAG_TY + 2.0 * g.ext_h[i]) * (g.ext[i] == 0 ? 1.0 : 4.0);
    return per_box + (double)DAG_TX * DAG_TY * 4.0 * g.outs.size();
}

int group_index(int n, int a0, int b0) { return a0 * n - a0 * (a0 - 1) / 2 + (b0 - a0); }  // 0-based first/last

int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

struct Geo {
    int64_t W, H, T, pitch, plane;
};
Geo geo_of(const kf_dag *d, int64_t W, int64_t H, int64_t T)
{
    Geo g{W, H, T, rup(W, 8), 0};
    g.plane = g.pitch * H * T;
    return g;
}

kf_status launch_plan(const GroupPlan &g, const kf_video *v, float *maps, const Geo &geo, float *out, int64_t opitch,
                      int out_node, cudaStream_t s)
{
    const size_t smem = (size_t)g.smem_bytes;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(dag_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DAG_SMEM_LIMIT) !=
            cudaSuccess)
            return KF_ECUDA;
        attr_set = true;
    }
    dim3 grid((unsigned)((v->W + DAG_TX - 1) / DAG_TX), (unsigned)((v->H + DAG_TY - 1) / DAG_TY), (unsigned)v->T);
    dag_group_kernel<<<grid, DAG_THREADS, smem, s>>>(g.prog, v->frames, v->pitch, maps, geo.plane, geo.pitch, out, opitch,
                                                     out_node, (int)v->W, (int)v->H);
    return cudaGetLastError() == cudaSuccess ? KF_OK : KF_ECUDA;
}

// features of a fused group for the learned cost model (per output pixel where relevant)
void features_of(const kf_dag *d, const GroupPlan &g, uint32_t members, int64_t W, int64_t H, int64_t T, float *f)
{
    const double tile = (double)DAG_TX * DAG_TY;
    int n_st = 0, n_sten = 0, sum_r = 0, hmax = 0;
    double compute = 0;
    for (int j = 1; j <= d->n; ++j) {
        if (!has(members, j) || g.halo[j] < 0) continue;
        const kf_gstage &s = d->st[j - 1];
        const int r = stage_radius(s);
        ++n_st;
        n_sten += r > 0;
        sum_r += r;
        const double area = (DAG_TX + 2.0 * g.halo[j]) * (DAG_TY + 2.0 * g.halo[j]) / tile;
        const double ops = s.kind == KF_G_STENCIL ? (2 * r + 1) * (2 * r + 1) : s.kind == KF_G_MAX3 ? 9 : s.kind == KF_G_PRODUCT ? 3 : 2;
        compute += area * ops;
    }
    double bytes_in = 0;
    for (size_t i = 0; i < g.ext.size(); ++i) {
        hmax = std::max(hmax, g.ext_h[i]);
        bytes_in += (DAG_TX + 2.0 * g.ext_h[i]) * (DAG_TY + 2.0 * g.ext_h[i]) / tile * (g.ext[i] == 0 ? 1.0 : 4.0);
    }
    f[0] = (float)n_st;
    f[1] = (float)n_sten;
    f[2] = (float)hmax;
    f[3] = (float)sum_r;
    f[4] = (float)bytes_in;
    f[5] = (float)(4.0 * g.outs.size());
    f[6] = (float)(g.smem_bytes / 1024.0);
    f[7] = (float)g.peak_slots;
    f[8] = (float)compute;
    f[9] = (float)g.ext.size();
    f[10] = (float)g.outs.size();
    f[11] = (float)std::log((double)W * H * T);
}

void features(const kf_dag *d, int a, int b, int64_t W, int64_t H, int64_t T, float *f)
{
    features_of(d, plan_group(d, a, b), range_mask(a, b), W, H, T, f);
}

// traffic (bytes) of the plan (cuts, X) and the largest on-chip bytes of its groups
double xplan_traffic(const kf_dag *d, uint32_t cuts, uint32_t X, double tiles, double *max_onchip)
{
    double t = 0, m = 0;
    int a = 1;
    for (int b = 1; b <= d->n; ++b) {
        if (b < d->n && !(cuts >> (b - 1) & 1)) continue;
        const GroupPlan g = plan_members(d, members_of(d, a, b, X), stores_of(d, a, b, X));
        t += tiles * tile_traffic(g);
        m = std::max(m, g.smem_bytes);
        a = b + 1;
    }
    *max_onchip = m;
    return t;
}

// Cost of a group under the planner's model: Sec. VI-D traffic, or the learned model's
// predicted time (memoised per group program: members and stores fix it).
struct PlanCost {
    const kf_dag *d;
    int64_t W, H, T;
    double tiles, limit;
    kf_ctx *model;  // nullptr: traffic
    std::unordered_map<uint64_t, double> memo;
    double operator()(int a, int b, uint32_t X)
    {
        const uint32_t mem = members_of(d, a, b, X), outs = stores_of(d, a, b, X);
        const uint64_t key = (uint64_t)mem << 32 | outs;
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
        const GroupPlan g = plan_members(d, mem, outs);
        double c = INFINITY;
        if (g.smem_bytes <= limit) {
            if (!model) {
                c = tiles * tile_traffic(g);
            } else {
                float f[KF_NFEAT], ms = 0.f;
                features_of(d, g, mem, W, H, T, f);
                if (kf::predict_group_ms(model, f, &ms) == KF_OK) c = ms;
            }
        }
        memo.emplace(key, c);
        return c;
    }
};

// The cheapest contiguous partition for a fixed inline set X (each group's cost depends
// only on its range and X, so the dynamic program over cut points is exact).
double best_cuts(const kf_dag *d, uint32_t X, PlanCost &cost, uint32_t *cuts)
{
    const int n = d->n;
    std::vector<double> best(n + 1, INFINITY);
    std::vector<int> from(n + 1, -1);
    best[0] = 0;
    for (int j = 1; j <= n; ++j)
        for (int i = 0; i < j; ++i) {
            if (!std::isfinite(best[i])) continue;
            const double c = best[i] + cost(i + 1, j, X);
            if (c < best[j]) {
                best[j] = c;
                from[j] = i;
            }
        }
    uint32_t m = 0;
    if (std::isfinite(best[n]))
        for (int j = n; j > 0; j = from[j])
            if (from[j] > 0) m |= 1u << (from[j] - 1);
    *cuts = m;
    return best[n];
}

bool valid_inline(const kf_dag *d, uint32_t X) { return d->n >= 32 || (X >> (d->n - 1)) == 0; }

}  // namespace

extern "C" {

kf_status kf_dag_create(kf_ctx *ctx, const kf_gstage *stages, int n, kf_dag **out)
{
    if (!ctx || !stages || !out || n < 1 || n > KF_DAG_MAX_STAGES) return KF_EINVAL;
    *out = nullptr;
    for (int i = 1; i <= n; ++i) {
        const kf_gstage &s = stages[i - 1];
        if (s.kind < KF_G_AFFINE || s.kind > KF_G_MAX3) return KF_EINVAL;
        if (s.in1 < 0 || s.in1 >= i) return KF_EINVAL;
        if (s.kind == KF_G_PRODUCT && (s.in2 < 0 || s.in2 >= i)) return KF_EINVAL;
        if (s.kind == KF_G_STENCIL && (s.radius < 0 || s.radius > 3)) return KF_EINVAL;
        if (!std::isfinite(s.a) || !std::isfinite(s.b)) return KF_EINVAL;
    }
    kf_dag *d = new (std::nothrow) kf_dag;
    if (!d) return KF_ENOMEM;
    d->device = kf::ctx_device(ctx);
    d->n = n;
    d->st.assign(stages, stages + n);
    d->cons.assign(n + 1, {});
    for (int i = 1; i <= n; ++i) {
        d->cons[stages[i - 1].in1].push_back(i);
        if (stages[i - 1].kind == KF_G_PRODUCT && stages[i - 1].in2 != stages[i - 1].in1) d->cons[stages[i - 1].in2].push_back(i);
    }
    *out = d;
    return KF_OK;
}

kf_status kf_dag_destroy(kf_dag *d)
{
    delete d;
    return KF_OK;
}

kf_status kf_dag_group_info(const kf_dag *d, int first, int last, int64_t W, int64_t H, int64_t T, float *features_out,
                            double *onchip_bytes, double *traffic_bytes)
{
    if (!d || first < 0 || last < first || last >= d->n || W <= 0 || H <= 0 || T <= 0) return KF_EINVAL;
    const GroupPlan g = plan_group(d, first + 1, last + 1);
    if (features_out) features(d, first + 1, last + 1, W, H, T, features_out);
    if (onchip_bytes) *onchip_bytes = g.smem_bytes;
    if (traffic_bytes) *traffic_bytes = (double)W * H * T / ((double)DAG_TX * DAG_TY) * tile_traffic(g);
    return KF_OK;
}

kf_status kf_dag_plan(const kf_dag *d, const double *group_cost, uint32_t *cuts, double *cost)
{
    if (!d || !group_cost || !cuts) return KF_EINVAL;
    const int n = d->n;
    std::vector<double> best(n + 1, INFINITY);
    std::vector<int> from(n + 1, -1);
    best[0] = 0;
    for (int j = 1; j <= n; ++j)
        for (int i = 0; i < j; ++i) {
            const double c = group_cost[group_index(n, i, j - 1)];
            if (!std::isfinite(best[i]) || !std::isfinite(c) || c < 0) continue;
            if (best[i] + c < best[j]) {
                best[j] = best[i] + c;
                from[j] = i;
            }
        }
    if (!std::isfinite(best[n])) return KF_ESMEM;
    uint32_t m = 0;
    for (int j = n; j > 0; j = from[j])
        if (from[j] > 0) m |= 1u << (from[j] - 1);
    *cuts = m;
    if (cost) *cost = best[n];
    return KF_OK;
}

kf_status kf_dag_workspace_bytes(const kf_dag *d, int64_t W, int64_t H, int64_t T, size_t *bytes)
{
    if (!d || !bytes || T <= 0 || !kf::volume_ok(W, H, T)) return KF_EINVAL;
    const Geo g = geo_of(d, W, H, T);
    *bytes = (size_t)(g.plane * 4) * (size_t)(d->n + 1);
    return KF_OK;
}

kf_status kf_dag_run(kf_dag *d, uint32_t cuts, const kf_video *v, float *out, int64_t out_pitch, void *ws,
                     size_t ws_bytes, void *stream)
{
    if (!d || !v || !out) return KF_EINVAL;
    if (d->device < 0) return KF_ESTATE;
    if (d->n < 32 && (cuts >> (d->n - 1))) return KF_EINVAL;
    if (v->W <= 0 || v->H <= 0 || v->T <= 0 || !v->frames || v->pitch < v->W || out_pitch < v->W) return KF_EINVAL;
    if (v->T > 65535 || v->H > (1 << 30)) return KF_EINVAL;
    size_t need = 0;
    if (kf_dag_workspace_bytes(d, v->W, v->H, v->T, &need) != KF_OK) return KF_EINVAL;
    if (!ws || ws_bytes < need) return KF_ENOMEM;
    kf::DeviceScope dev_scope(d->device);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
    const Geo geo = geo_of(d, v->W, v->H, v->T);
    int a = 1;
    for (int b = 1; b <= d->n; ++b) {
        if (b < d->n && !(cuts >> (b - 1) & 1)) continue;
        const GroupPlan g = plan_group(d, a, b);
        if (!g.feasible) return KF_ESMEM;
        kf_status st = launch_plan(g, v, static_cast<float *>(ws), geo, out, out_pitch, d->n, static_cast<cudaStream_t>(stream));
        if (st != KF_OK) return st;
        a = b + 1;
    }
    return KF_OK;
}

kf_status kf_dag_time_groups(kf_dag *d, const kf_video *v, float *out, int64_t out_pitch, void *ws, size_t ws_bytes,
                             int reps, void *stream, float *ms)
{
    if (!d || !v || !ms || reps < 1) return KF_EINVAL;
    const int n = d->n;
    // materialise every node once (no fusion), so that any group finds its inputs
    kf_status st = kf_dag_run(d, n > 1 ? (uint32_t)((1ull << (n - 1)) - 1) : 0u, v, out, out_pitch, ws, ws_bytes, stream);
    if (st != KF_OK) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Geo geo = geo_of(d, v->W, v->H, v->T);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return KF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KF_ECUDA;
    }
    for (int a = 1; a <= n && st == KF_OK; ++a)
        for (int b = a; b <= n && st == KF_OK; ++b) {
            const GroupPlan g = plan_group(d, a, b);
            float &slot = ms[group_index(n, a - 1, b - 1)];
            if (!g.feasible) {
                slot = -1.0f;
                continue;
            }
            st = launch_plan(g, v, static_cast<float *>(ws), geo, out, out_pitch, n, s);  // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == KF_OK; ++r)
                st = launch_plan(g, v, static_cast<float *>(ws), geo, out, out_pitch, n, s);
            cudaEventRecord(e1, s);
            float t = 0;
            if (st == KF_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
                st = KF_ECUDA;
            slot = t / reps;
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

kf_status kf_dag_xplan_traffic(const kf_dag *d, uint32_t cuts, uint32_t inline_mask, int64_t W, int64_t H, int64_t T,
                               double *bytes, double *max_onchip)
{
    if (!d || !bytes || W <= 0 || H <= 0 || T <= 0 || !valid_inline(d, inline_mask)) return KF_EINVAL;
    if (d->n < 32 && (cuts >> (d->n - 1))) return KF_EINVAL;
    double m = 0;
    *bytes = xplan_traffic(d, cuts, inline_mask, (double)W * H * T / ((double)DAG_TX * DAG_TY), &m);
    if (max_onchip) *max_onchip = m;
    return KF_OK;
}

kf_status kf_dag_plan_recompute(const kf_dag *d, int64_t W, int64_t H, int64_t T, double onchip_limit, kf_ctx *model,
                                uint32_t *cuts, uint32_t *inline_mask, double *cost_out)
{
    if (!d || !cuts || !inline_mask || W <= 0 || H <= 0 || T <= 0) return KF_EINVAL;
    if (model) {  // a model that is not trained (or set) predicts nothing
        float f[KF_NFEAT] = {}, ms = 0.f;
        if (kf::predict_group_ms(model, f, &ms) != KF_OK) return KF_ESTATE;
    }
    const int n = d->n;
    PlanCost cost{d, W, H, T, (double)W * H * T / ((double)DAG_TX * DAG_TY),
                  onchip_limit > 0 && onchip_limit < DAG_SMEM_LIMIT ? onchip_limit : DAG_SMEM_LIMIT, model, {}};
    uint32_t best_c = 0, best_x = 0;
    double best = best_cuts(d, 0, cost, &best_c);
    if (n - 1 <= KF_DAG_EXACT_INLINE) {
        // every inline set of the n - 1 non-output nodes in increasing order; only a
        // strictly cheaper plan replaces the best, so the contiguous plan wins ties
        for (uint32_t X = 1; X < (1u << (n - 1)); ++X) {
            uint32_t c = 0;
            const double t = best_cuts(d, X, cost, &c);
            if (t < best) {
                best = t;
                best_c = c;
                best_x = X;
            }
        }
    } else {
        // hill climbing over single-node toggles from the contiguous optimum
        for (bool improved = true; improved;) {
            improved = false;
            uint32_t step_x = best_x, step_c = best_c;
            double step = best;
            for (int j = 1; j < n; ++j) {
                uint32_t c = 0;
                const uint32_t X = best_x ^ (1u << (j - 1));
                const double t = best_cuts(d, X, cost, &c);
                if (t < step) {
                    step = t;
                    step_x = X;
                    step_c = c;
                }
            }
            if (step < best) {
                best = step;
                best_x = step_x;
                best_c = step_c;
                improved = true;
            }
        }
    }
    if (!std::isfinite(best)) return KF_ESMEM;
    *cuts = best_c;
    *inline_mask = best_x;
    if (cost_out) *cost_out = best;
    return KF_OK;
}

kf_status kf_dag_run_x(kf_dag *d, uint32_t cuts, uint32_t inline_mask, const kf_video *v, float *out, int64_t out_pitch,
                       void *ws, size_t ws_bytes, void *stream)
{
    if (!d || !v || !out || !valid_inline(d, inline_mask)) return KF_EINVAL;
    if (d->device < 0) return KF_ESTATE;
    if (d->n < 32 && (cuts >> (d->n - 1))) return KF_EINVAL;
    if (v->W <= 0 || v->H <= 0 || v->T <= 0 || !v->frames || v->pitch < v->W || out_pitch < v->W) return KF_EINVAL;
    if (v->T > 65535 || v->H > (1 << 30)) return KF_EINVAL;
    size_t need = 0;
    if (kf_dag_workspace_bytes(d, v->W, v->H, v->T, &need) != KF_OK) return KF_EINVAL;
    if (!ws || ws_bytes < need) return KF_ENOMEM;
    std::vector<GroupPlan> plans;
    int a = 1;
    for (int b = 1; b <= d->n; ++b) {  // every group checked before anything is enqueued
        if (b < d->n && !(cuts >> (b - 1) & 1)) continue;
        plans.push_back(plan_members(d, members_of(d, a, b, inline_mask), stores_of(d, a, b, inline_mask)));
        if (!plans.back().feasible) return KF_ESMEM;
        a = b + 1;
    }
    kf::DeviceScope dev_scope(d->device);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
    const Geo geo = geo_of(d, v->W, v->H, v->T);
    for (const GroupPlan &g : plans) {
        const kf_status st =
            launch_plan(g, v, static_cast<float *>(ws), geo, out, out_pitch, d->n, static_cast<cudaStream_t>(stream));
        if (st != KF_OK) return st;
    }
    return KF_OK;
}

kf_status kf_dag_time_xgroups(kf_dag *d, const kf_video *v, float *out, int64_t out_pitch, void *ws, size_t ws_bytes,
                              const int32_t *groups, int count, int reps, void *stream, float *ms, float *features)
{
    if (!d || !v || !groups || count < 0 || !ms || reps < 1) return KF_EINVAL;
    const int n = d->n;
    for (int g = 0; g < count; ++g) {
        const int a = groups[3 * g], b = groups[3 * g + 1];
        const uint32_t X = (uint32_t)groups[3 * g + 2];
        if (a < 0 || b < a || b >= n || !valid_inline(d, X)) return KF_EINVAL;
    }
    // materialise every node once (no fusion), so that any group finds its inputs
    kf_status st = kf_dag_run(d, n > 1 ? (uint32_t)((1ull << (n - 1)) - 1) : 0u, v, out, out_pitch, ws, ws_bytes, stream);
    if (st != KF_OK) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Geo geo = geo_of(d, v->W, v->H, v->T);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return KF_ECUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return KF_ECUDA;
    }
    for (int g = 0; g < count && st == KF_OK; ++g) {
        const int a = groups[3 * g] + 1, b = groups[3 * g + 1] + 1;
        const uint32_t X = (uint32_t)groups[3 * g + 2];
        const uint32_t mem = members_of(d, a, b, X);
        const GroupPlan gp = plan_members(d, mem, stores_of(d, a, b, X));
        if (features) features_of(d, gp, mem, v->W, v->H, v->T, features + (size_t)g * KF_NFEAT);
        if (!gp.feasible) {
            ms[g] = -1.0f;
            continue;
        }
        st = launch_plan(gp, v, static_cast<float *>(ws), geo, out, out_pitch, n, s);  // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == KF_OK; ++r) st = launch_plan(gp, v, static_cast<float *>(ws), geo, out, out_pitch, n, s);
        cudaEventRecord(e1, s);
        float t = 0;
        if (st == KF_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
            st = KF_ECUDA;
        ms[g] = t / reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // extern "C"
