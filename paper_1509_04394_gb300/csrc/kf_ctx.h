// kf_ctx.h -- the context object behind the opaque kf_ctx handle (library-internal).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/kfuse.h"

namespace kf {
struct CostModel;                   // kf_mlp.cu
void costmodel_free(kf_ctx *ctx);   // kf_mlp.cu

// The volumes the library sizes workspaces for: sides of 1..2^30 pixels, 0..2^31-1 frames
// and at most 2^46 pixels in all (far beyond device memory), so that no workspace byte
// count (a few tens of bytes per pixel at most) can overflow 64 bits.
inline bool volume_ok(int64_t W, int64_t H, int64_t T)
{
    if (W <= 0 || H <= 0 || T < 0 || W > (1 << 30) || H > (1 << 30) || T > 0x7fffffffLL) return false;
    return T == 0 || W * H <= ((int64_t)1 << 46) / T;
}
}  // namespace kf

struct kf_ctx {
    int device = -1;
    int precision = KF_PREC_F32;
    int chunk_rows = 200;
    int host_chunk_rows = 0;  // tile height of kf_track_host's chunk launches (0: chunk_rows)
    unsigned wait_polls = 1u << 22;  // kf::WAIT_POLLS unless kf_set_wait_polls lowered it
    int last_cuda = 0;
    int *d_err = nullptr;  // device error word of the bounded waits (4 bytes, owned)
    std::vector<kf_stage_desc> stages;
    kf::CostModel *cm = nullptr;  // learned cost model (host parameters), owned
    // kernel timing: recorded (kind, start, end) event triples, and spare events (owned)
    struct Timed { int kind; cudaEvent_t a, b; };
    bool timing = false;
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> spare_events;
    // events made when timing is switched on: pairs for 512 launches, more on demand
    static constexpr size_t TIMING_EVENTS = 1024;
    // kf_track_host: the copy-in, compute and copy-out streams and their event rings (owned)
    static constexpr int N_RING = 3;
    cudaStream_t s_in = nullptr, s_out = nullptr, s_comp[N_RING] = {}, s_trk[N_RING] = {};
    cudaEvent_t ev_in[N_RING] = {}, ev_comp[N_RING] = {}, ev_chain[N_RING] = {}, ev_edge = nullptr;
    // kf_track_host with packed masks: device staging of the packed chunks (owned)
    uint8_t *pack_buf = nullptr;
    size_t pack_bytes = 0;
};
