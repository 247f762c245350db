// kf_static.cu -- kf_run_static: the partitioned chain with its workspace in a fixed,
// library-owned device array, for callers that must not allocate device memory.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library
// holds its own KF_STATIC_WORKSPACE_BYTES copy until the process exits. On the host,
// the name g_static_ws is only a shadow symbol, not a device address: passing it to a
// kernel would fault or, where the GPU can reach host memory, silently use the wrong
// memory. The device address of each GPU's copy is therefore looked up once per device,
// with that device current, by cudaGetSymbolAddress, and only that address is handed to
// the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/kfuse.h"
#include "kf_device.h"

namespace kf {
int ctx_device(const kf_ctx *ctx);  // kf_api.cu
}

namespace {

static __device__ __align__(256) unsigned char g_static_ws[KF_STATIC_WORKSPACE_BYTES];

constexpr int MAX_DEVICES = 64;
void *g_ws_addr[MAX_DEVICES];  // device address of g_static_ws per device, once looked up
std::mutex g_ws_mu;

// The set-up: with `device` current, resolve the device address of its copy (first call
// on that device only).
cudaError_t static_workspace(int device, void **addr)
{
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (!g_ws_addr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess) return e;
        g_ws_addr[device] = p;
    }
    *addr = g_ws_addr[device];
    return cudaSuccess;
}

}  // namespace

extern "C" kf_status kf_run_static(kf_ctx *ctx, uint32_t cuts, const kf_video *video, const kf_corners *out,
                                   void *stream)
{
    if (!ctx || !video) return KF_EINVAL;
    const int device = kf::ctx_device(ctx);
    if (device < 0) return KF_ESTATE;
    if (device >= MAX_DEVICES) return KF_EUNSUPPORTED;
    size_t need = 0;
    kf_status s = kf_workspace_bytes(ctx, cuts, video->W, video->H, video->T, &need);
    if (s != KF_OK) return s;
    if (need > (size_t)KF_STATIC_WORKSPACE_BYTES) return KF_ENOMEM;  // larger than the fixed array
    kf::DeviceScope dev_scope(device);
    if (dev_scope.status() != cudaSuccess) return KF_ECUDA;
    void *ws = nullptr;
    if (static_workspace(device, &ws) != cudaSuccess) return KF_ECUDA;
    // Every map the groups write in the workspace is written in full before it is read,
    // so the previous call's contents never need clearing; the per-frame counts live in
    // the caller's buffer and kf_run zeroes them.
    return kf_run(ctx, cuts, video, out, ws, (size_t)KF_STATIC_WORKSPACE_BYTES, stream);
}
