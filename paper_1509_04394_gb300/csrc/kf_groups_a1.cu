// kf_groups_a1.cu -- fused group kernels whose first stage is stage 1 (one TU per first
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

// the persistent batch of fully fused chains over many videos
int launch_batch_chain(const GroupParams *videos, const int64_t *item_begin, int n_videos, unsigned long long *queue,
                       bool cand, unsigned grid, int sm_split, void *stream)
{
    if (cand)
        batch_kernel<true><<<grid, 32 * WARPS_PER_BLOCK, SmemPlan<1, 8, false, true>::BYTES, static_cast<cudaStream_t>(stream)>>>(
            videos, item_begin, n_videos, queue, sm_split);
    else
        batch_kernel<false><<<grid, 32 * WARPS_PER_BLOCK, SmemPlan<1, 8, false, false>::BYTES, static_cast<cudaStream_t>(stream)>>>(
            videos, item_begin, n_videos, queue, sm_split);
    return (int)cudaGetLastError();
}

int batch_chain_blocks_per_sm(bool cand)
{
    int n = 0;
    cudaError_t e = cand ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<true>, 32 * WARPS_PER_BLOCK,
                                                                         SmemPlan<1, 8, false, true>::BYTES)
                         : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<false>, 32 * WARPS_PER_BLOCK,
                                                                         SmemPlan<1, 8, false, false>::BYTES);
    return e == cudaSuccess ? n : 0;
}

// the fully fused chain that also lists every frame's corners for the tracking stage
int launch_chain_with_candidates(const GroupParams &p, unsigned grid, void *stream)
{
    group_kernel<1, 8, false, true><<<grid, 32 * WARPS_PER_BLOCK, SmemPlan<1, 8, false, true>::BYTES,
                                      static_cast<cudaStream_t>(stream)>>>(p);
    return (int)cudaGetLastError();
}

// the same with FP16 inter-stage tiles (the box's ring in FP16, see run_job)
int launch_chain_with_candidates_tiles(const GroupParams &p, unsigned grid, void *stream)
{
    group_kernel<1, 8, true, true, true><<<grid, 32 * WARPS_PER_BLOCK, SmemPlan<1, 8, true, true>::BYTES,
                                           static_cast<cudaStream_t>(stream)>>>(p);
    return (int)cudaGetLastError();
}

LaunchFn launcher_a1(int B, int f16)
{
    switch (B) {
    case 1: return f16 ? launch<1, 1, true> : launch<1, 1, false>;
    case 2: return f16 ? launch<1, 2, true> : launch<1, 2, false>;
    case 3: return f16 ? launch<1, 3, true> : launch<1, 3, false>;
    case 4: return f16 ? launch<1, 4, true> : launch<1, 4, false>;
    case 5: return f16 ? launch<1, 5, true> : launch<1, 5, false>;
    case 6: return f16 ? launch<1, 6, true> : launch<1, 6, false>;
    case 7: return f16 ? launch<1, 7, true> : launch<1, 7, false>;
    case 8: return f16 == 2 ? launch<1, 8, true, true> : f16 ? launch<1, 8, true> : launch<1, 8, false>;
    default: return nullptr;
    }
}
}  // namespace kf
