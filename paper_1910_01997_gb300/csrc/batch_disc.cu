// Batched Gauss-Newton kernel of circular surfels (plans with surfel_radius): one warp per surfel,
// up to kBatchDiscPPL disc pixels per lane.
#include "batch_impl.cuh"

namespace sgn {

__global__ void __launch_bounds__(kBatchBlock, 2) k_gn_batch_disc(const PlanParams* __restrict__ plans,
                                                               const WorkItem* __restrict__ items, int n_items,
                                                               int* __restrict__ counter, int iters, int max_frames) {
    __shared__ PlanParams spp[kBatchWarps];
    extern __shared__ float4 sdyn[];
    batch_loop<kBatchDisc, 0>(plans, items, n_items, counter, iters, max_frames, spp, reinterpret_cast<float*>(sdyn));
}

namespace {
LaunchAttrs g_disc_attrs;
}

int batch_blocks_per_sm_disc(int block_threads, int max_frames) {
    return batch_blocks_per_sm_of(k_gn_batch_disc, g_disc_attrs, block_threads, max_frames);
}

int launch_gn_batch_disc(const PlanParams* d_plans, const WorkItem* d_items, int n_items, int* d_counter, int iters,
                         int grid, int block_threads, int max_frames, cudaStream_t st) {
    return launch_batch_kernel(k_gn_batch_disc, g_disc_attrs, d_plans, d_items, n_items, d_counter, iters, grid,
                               block_threads, max_frames, st);
}

}  // namespace sgn
