// kf_groups_a2.cu -- fused group kernels whose first stage is stage 2 (one TU per first
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

LaunchFn launcher_a2(int B, int f16)
{
    switch (B) {
    case 2: return f16 ? launch<2, 2, __half> : launch<2, 2, float>;
    case 3: return f16 ? launch<2, 3, __half> : launch<2, 3, float>;
    case 4: return f16 ? launch<2, 4, __half> : launch<2, 4, float>;
    case 5: return f16 ? launch<2, 5, __half> : launch<2, 5, float>;
    case 6: return f16 ? launch<2, 6, __half> : launch<2, 6, float>;
    case 7: return f16 ? launch<2, 7, __half> : launch<2, 7, float>;
    case 8: return f16 ? launch<2, 8, __half> : launch<2, 8, float>;
    default: return nullptr;
    }
}
}  // namespace kf
