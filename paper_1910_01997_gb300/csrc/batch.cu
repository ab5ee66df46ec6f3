// Persistent batched Gauss-Newton: many keyframe problems (any size, patch, frame count and
// texel dtype) in one launch.  Each warp pulls (plan, surfel range) work items from a device
// work list through an atomic counter and runs the same per-surfel solver as the plain launch
// (seeding, iterations, final cost, depth map).  The counter is reset by a memset on the same
// stream before every launch; there is no waiting on other warps or blocks.
#include <cuda_runtime.h>

#include "gn_impl.cuh"

namespace sgn {

constexpr int kBatchBlock = 256;
constexpr int kBatchWarps = kBatchBlock / 32;

__host__ __device__ constexpr int batch_lanes(int variant, int P) {
    return P == 16 ? 32 : (P == 8 ? (variant == 0 ? 16 : 32) : (variant == 0 ? 8 : 16));
}

int lanes_for_patch(int variant, int P) { return batch_lanes(variant, P); }

template <int P, int G, int DT>
__device__ __forceinline__ void run_chunk(const PlanParams* pp, int first, int count, int lane, int iters,
                                          float* ref, int group_words) {
    constexpr int SPW = 32 / G;  // surfels per warp step
    const int end = first + count;
    for (int base = first; base < end; base += SPW) {
        const int s = base + lane / G;
        // passes of at most 4 pixels per lane keep every patch size within the kernel's 128 registers;
        // all four pixels of a pass gather before use (two at a time in the plain launch: measured
        // best for each kernel on the benchmark workloads)
        gn_surfel<P, G, DT, false, 4, 0, false, 4>(pp, s < end ? s : pp->S, lane % G, iters, kModeSolve,
                                                    ref + (lane / G) * group_words);
        __syncwarp();
    }
}

template <int V, int DT>
__device__ __forceinline__ void dispatch_patch(const PlanParams* pp, const WorkItem& w, int lane, int iters,
                                               float* ref, int group_words) {
    switch (pp->P) {
        case 4: run_chunk<4, batch_lanes(V, 4), DT>(pp, w.first, w.count, lane, iters, ref, group_words); break;
        case 8: run_chunk<8, batch_lanes(V, 8), DT>(pp, w.first, w.count, lane, iters, ref, group_words); break;
        case 16: run_chunk<16, batch_lanes(V, 16), DT>(pp, w.first, w.count, lane, iters, ref, group_words); break;
        default: break;
    }
}

// Groups per warp at most (8 lanes per surfel: 4x4 tiles in variant 0).
constexpr int kBatchGroups = 4;

// Dynamic shared memory: per warp, kBatchGroups frame scratches of max_frames frames.
int batch_scratch_bytes(int max_frames) { return kBatchWarps * kBatchGroups * group_scratch_words(max_frames) * 4; }

template <int V>
__global__ void __launch_bounds__(kBatchBlock, 2) k_gn_batch(const PlanParams* __restrict__ plans,
                                                          const WorkItem* __restrict__ items, int n_items,
                                                          int* __restrict__ counter, int iters, int max_frames) {
    __shared__ PlanParams spp[kBatchWarps];
    extern __shared__ float4 sdyn[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group_words = group_scratch_words(max_frames);
    float* wref = reinterpret_cast<float*>(sdyn) + warp * kBatchGroups * group_words;
    PlanParams* my = &spp[warp];
    int cur = -1;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const WorkItem w = items[it];
        if (w.plan != cur) {
            __syncwarp();
            const int* src = reinterpret_cast<const int*>(plans + w.plan);
            int* dst = reinterpret_cast<int*>(my);
            for (int i = lane; i < int(sizeof(PlanParams) / 4); i += 32) dst[i] = __ldg(src + i);
            __syncwarp();
            cur = w.plan;
        }
        switch (my->dtype) {
            case SGN_F32: dispatch_patch<V, SGN_F32>(my, w, lane, iters, wref, group_words); break;
            case SGN_F16: dispatch_patch<V, SGN_F16>(my, w, lane, iters, wref, group_words); break;
            case SGN_BF16: dispatch_patch<V, SGN_BF16>(my, w, lane, iters, wref, group_words); break;
            case SGN_F16G: dispatch_patch<V, SGN_F16G>(my, w, lane, iters, wref, group_words); break;
            case SGN_BF16G: dispatch_patch<V, SGN_BF16G>(my, w, lane, iters, wref, group_words); break;
            default: break;
        }
    }
}

LaunchAttrs g_batch_attrs[2];

// Dynamic shared-memory limit and carveout of variant V on the current device for max_frames.
static cudaError_t batch_attributes(int variant, int max_frames) {
    const int smem = batch_scratch_bytes(max_frames), max_bytes = batch_scratch_bytes(kMaxFrames);
    return variant == 0 ? configure_launch(k_gn_batch<0>, g_batch_attrs[0], max_bytes, smem, 2)
                        : configure_launch(k_gn_batch<1>, g_batch_attrs[1], max_bytes, smem, 2);
}

int batch_blocks_per_sm(int variant, int block_threads, int max_frames) {
    if (max_frames < 1 || max_frames > kMaxFrames || batch_attributes(variant, max_frames) != cudaSuccess) return 0;
    int n = 0;
    const size_t smem = batch_scratch_bytes(max_frames);
    cudaError_t e = variant == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gn_batch<0>, block_threads, smem)
                                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_gn_batch<1>, block_threads, smem);
    return e == cudaSuccess ? n : 0;
}

int launch_gn_batch(const PlanParams* d_plans, const WorkItem* d_items, int n_items, int* d_counter, int iters,
                    int variant, int grid, int block_threads, int max_frames, void* stream) {
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (block_threads != kBatchBlock || max_frames < 1 || max_frames > kMaxFrames) return int(cudaErrorInvalidConfiguration);
    cudaError_t e = batch_attributes(variant, max_frames);
    if (e != cudaSuccess) return int(e);
    e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return int(e);
    const size_t smem = batch_scratch_bytes(max_frames);
    if (variant == 0)
        k_gn_batch<0><<<grid, block_threads, smem, st>>>(d_plans, d_items, n_items, d_counter, iters, max_frames);
    else
        k_gn_batch<1><<<grid, block_threads, smem, st>>>(d_plans, d_items, n_items, d_counter, iters, max_frames);
    return int(cudaGetLastError());
}

}  // namespace sgn
