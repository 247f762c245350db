// kf_groups_a8.cu -- fused group kernels whose first stage is stage 8 (one TU per first
// stage so that the 72 instantiations compile in parallel).
#include <cuda_runtime.h>

#include "kf_chain.cuh"

namespace kf {
namespace {
template <int A, int B, bool F16, bool TILES = false>
int launch(const GroupParams &p, unsigned grid, void *stream)
{
    group_kernel<A, B, F16, false, TILES>
        <<<grid, 32 * WARPS_PER_BLOCK, SmemPlan<A, B, F16>::BYTES, static_cast<cudaStream_t>(stream)>>>(p);
    return (int)cudaGetLastError();
}
}  // namespace

LaunchFn launcher_a8(int B, int f16)
{
    switch (B) {
    case 8: return f16 ? launch<8, 8, true> : launch<8, 8, false>;
    default: return nullptr;
    }
}
}  // namespace kf
