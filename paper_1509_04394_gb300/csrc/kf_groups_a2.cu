// kf_groups_a2.cu -- fused group kernels whose first stage is stage 2 (one TU per first
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

LaunchFn launcher_a2(int B, int f16)
{
    switch (B) {
    case 2: return f16 ? launch<2, 2, true> : launch<2, 2, false>;
    case 3: return f16 ? launch<2, 3, true> : launch<2, 3, false>;
    case 4: return f16 ? launch<2, 4, true> : launch<2, 4, false>;
    case 5: return f16 ? launch<2, 5, true> : launch<2, 5, false>;
    case 6: return f16 ? launch<2, 6, true> : launch<2, 6, false>;
    case 7: return f16 ? launch<2, 7, true> : launch<2, 7, false>;
    case 8: return f16 == 2 ? launch<2, 8, true, true> : f16 ? launch<2, 8, true> : launch<2, 8, false>;
    default: return nullptr;
    }
}
}  // namespace kf
