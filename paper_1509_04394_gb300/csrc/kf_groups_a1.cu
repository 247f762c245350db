// kf_groups_a1.cu -- fused group kernels whose first stage is stage 1 (one TU per first
// stage so that the 72 instantiations compile in parallel).
#include <cuda_runtime.h>

#include "kf_chain.cuh"

namespace kf {
namespace {
template <int A, int B, typename TM>
int launch(const GroupParams &p, unsigned grid, void *stream)
{
    group_kernel<A, B, TM><<<grid, 32 * WARPS_PER_BLOCK, 0, static_cast<cudaStream_t>(stream)>>>(p);
    return (int)cudaGetLastError();
}
}  // namespace

LaunchFn launcher_a1(int B, int f16)
{
    switch (B) {
    case 1: return f16 ? launch<1, 1, __half> : launch<1, 1, float>;
    case 2: return f16 ? launch<1, 2, __half> : launch<1, 2, float>;
    case 3: return f16 ? launch<1, 3, __half> : launch<1, 3, float>;
    case 4: return f16 ? launch<1, 4, __half> : launch<1, 4, float>;
    case 5: return f16 ? launch<1, 5, __half> : launch<1, 5, float>;
    case 6: return f16 ? launch<1, 6, __half> : launch<1, 6, float>;
    case 7: return f16 ? launch<1, 7, __half> : launch<1, 7, float>;
    case 8: return f16 ? launch<1, 8, __half> : launch<1, 8, float>;
    default: return nullptr;
    }
}
}  // namespace kf
