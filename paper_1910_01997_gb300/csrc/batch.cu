// Batched Gauss-Newton with fixed damping (square surfels), and the dispatch of the batch launches
// of every solver kind.
#include "batch_impl.cuh"

namespace sgn {

int lanes_for_patch(int variant, int P) { return batch_lanes(variant, P); }
int square_items(int P, int TX, int TY) { return square_blocks(TX, TY, kBatchBlock / batch_lanes(2, P)); }

template <int V>
__global__ void __launch_bounds__(kBatchBlock, 2) k_gn_batch(const PlanParams* __restrict__ plans,
                                                          const WorkItem* __restrict__ items, int n_items,
                                                          int* __restrict__ counter, int iters, int max_frames) {
    __shared__ PlanParams spp[kBatchWarps];
    extern __shared__ float4 sdyn[];
    if constexpr (V == 2) {
        __shared__ int s_item;
        batch_square_loop(plans, items, n_items, counter, iters, max_frames, spp, reinterpret_cast<float*>(sdyn), &s_item);
    } else {
        batch_loop<kBatchFixed, V>(plans, items, n_items, counter, iters, max_frames, spp, reinterpret_cast<float*>(sdyn));
    }
}

namespace {
LaunchAttrs g_fixed_attrs[3];
}

// The other kinds' kernels (batch_adaptive.cu, batch_disc.cu).
int batch_blocks_per_sm_adaptive(int block_threads, int max_frames);
int batch_blocks_per_sm_disc(int block_threads, int max_frames);
int launch_gn_batch_adaptive(const PlanParams*, const WorkItem*, int, int*, int, int, int, int, cudaStream_t);
int launch_gn_batch_disc(const PlanParams*, const WorkItem*, int, int*, int, int, int, int, cudaStream_t);

int batch_blocks_per_sm(int kind, int variant, int block_threads, int max_frames) {
    switch (kind) {
        case kBatchFixed:
            return variant == 0   ? batch_blocks_per_sm_of(k_gn_batch<0>, g_fixed_attrs[0], block_threads, max_frames)
                   : variant == 1 ? batch_blocks_per_sm_of(k_gn_batch<1>, g_fixed_attrs[1], block_threads, max_frames)
                                  : batch_blocks_per_sm_of(k_gn_batch<2>, g_fixed_attrs[2], block_threads, max_frames);
        case kBatchAdaptive: return batch_blocks_per_sm_adaptive(block_threads, max_frames);
        case kBatchDisc: return batch_blocks_per_sm_disc(block_threads, max_frames);
        default: return 0;
    }
}

int launch_gn_batch(int kind, const PlanParams* d_plans, const WorkItem* d_items, int n_items, int* d_counter, int iters,
                    int variant, int grid, int block_threads, int max_frames, void* stream) {
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (kind) {
        case kBatchFixed:
            if (variant == 0)
                return launch_batch_kernel(k_gn_batch<0>, g_fixed_attrs[0], d_plans, d_items, n_items, d_counter, iters, grid,
                                           block_threads, max_frames, st);
            if (variant == 1)
                return launch_batch_kernel(k_gn_batch<1>, g_fixed_attrs[1], d_plans, d_items, n_items, d_counter, iters, grid,
                                           block_threads, max_frames, st);
            return launch_batch_kernel(k_gn_batch<2>, g_fixed_attrs[2], d_plans, d_items, n_items, d_counter, iters, grid,
                                       block_threads, max_frames, st);
        case kBatchAdaptive:
            return launch_gn_batch_adaptive(d_plans, d_items, n_items, d_counter, iters, grid, block_threads, max_frames, st);
        case kBatchDisc:
            return launch_gn_batch_disc(d_plans, d_items, n_items, d_counter, iters, grid, block_threads, max_frames, st);
        default: return int(cudaErrorInvalidValue);
    }
}

}  // namespace sgn
