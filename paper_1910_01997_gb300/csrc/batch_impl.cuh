// Persistent batched Gauss-Newton (shared by the batch kernels of each solver kind): each warp pulls
// (plan, surfel range) work items from a device work list through an atomic counter and runs the
// same per-surfel solver as the plain launch (seeding, iterations, final cost, depth map).  The
// counter is reset by a memset on the same stream before every launch; there is no waiting on other
// warps or blocks.  A batch launches one kernel per solver kind present (fixed damping; the
// Marquardt schedule; circular surfels), each over its own contiguous range of the work list, so
// that no kernel carries the registers of another kind's solver.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "gn_impl.cuh"

namespace sgn {

constexpr int kBatchBlock = 256;
constexpr int kBatchWarps = kBatchBlock / 32;
// Groups per warp at most (8 lanes per surfel: 4x4 tiles in variant 0).
constexpr int kBatchGroups = 4;
// Circular surfels in a batch: up to this many disc pixels per lane (16 x 32 lanes = kMaxDiscPixels);
// passes past a plan's disc are skipped at run time.
constexpr int kBatchDiscPPL = 16;

// Lanes per surfel of the fixed-damping schedules: variants 0 (warp items) and 2 (square items) map
// P = 4 / 8 / 16 to 8 / 16 / 32 lanes, variant 1 to 16 / 32 / 32.
__host__ __device__ constexpr int batch_lanes(int variant, int P) {
    return P == 16 ? 32 : (P == 8 ? (variant == 1 ? 32 : 16) : (variant == 1 ? 16 : 8));
}

// Dynamic shared memory: per warp, kBatchGroups frame scratches of max_frames frames.
inline int batch_scratch_bytes(int max_frames) { return kBatchWarps * kBatchGroups * group_scratch_words(max_frames) * 4; }

// Lanes per surfel of a solver kind and schedule variant.
template <int KIND, int V, int P>
struct KindLanes {
    static constexpr int G = KIND == kBatchDisc ? 32 : batch_lanes(V, P);
};

template <int KIND, int V, int P, int DT>
__device__ __forceinline__ void run_chunk(const PlanParams* pp, int first, int count, int lane, int iters,
                                          float* ref, int group_words) {
    constexpr int G = KindLanes<KIND, V, P>::G;
    constexpr int SPW = 32 / G;  // surfels per warp step
    constexpr bool LMA = KIND == kBatchAdaptive;
    constexpr int DPPL = KIND == kBatchDisc ? kBatchDiscPPL : 0;
    const int end = first + count;
    for (int base = first; base < end; base += SPW) {
        const int s = base + lane / G;
        // passes of at most 4 pixels per lane keep every patch size within the kernel's 128 registers;
        // all four pixels of a pass gather before use
        gn_surfel<P, G, DT, false, 4, DPPL, LMA, 4>(pp, s < end ? s : pp->S, lane % G, iters, kModeSolve,
                                                     ref + (lane / G) * group_words);
        __syncwarp();
    }
}

template <int KIND, int V, int DT>
__device__ __forceinline__ void dispatch_patch(const PlanParams* pp, const WorkItem& w, int lane, int iters,
                                               float* ref, int group_words) {
    switch (pp->P) {
        case 4: run_chunk<KIND, V, 4, DT>(pp, w.first, w.count, lane, iters, ref, group_words); break;
        case 8: run_chunk<KIND, V, 8, DT>(pp, w.first, w.count, lane, iters, ref, group_words); break;
        case 16: run_chunk<KIND, V, 16, DT>(pp, w.first, w.count, lane, iters, ref, group_words); break;
        default: break;
    }
}

// The persistent loop of one batch kernel (all threads of the block).
template <int KIND, int V>
__device__ __forceinline__ void batch_loop(const PlanParams* __restrict__ plans, const WorkItem* __restrict__ items,
                                           int n_items, int* __restrict__ counter, int iters, int max_frames,
                                           PlanParams* spp, float* sdyn) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group_words = group_scratch_words(max_frames);
    float* wref = sdyn + warp * kBatchGroups * group_words;
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
            const int n = plan_words(__ldg(&plans[w.plan].F));
            for (int i = lane; i < n; i += 32) dst[i] = __ldg(src + i);
            __syncwarp();
            cur = w.plan;
        }
        switch (my->dtype) {
            case SGN_F32: dispatch_patch<KIND, V, SGN_F32>(my, w, lane, iters, wref, group_words); break;
            case SGN_F16: dispatch_patch<KIND, V, SGN_F16>(my, w, lane, iters, wref, group_words); break;
            case SGN_BF16: dispatch_patch<KIND, V, SGN_BF16>(my, w, lane, iters, wref, group_words); break;
            case SGN_F16G: dispatch_patch<KIND, V, SGN_F16G>(my, w, lane, iters, wref, group_words); break;
            case SGN_BF16G: dispatch_patch<KIND, V, SGN_BF16G>(my, w, lane, iters, wref, group_words); break;
            default: break;
        }
    }
}

// The persistent loop over square items (schedule variant 2, fixed damping): a whole block takes one
// item, a square of neighbouring tiles of one plan (the block's surfels of a plain launch,
// square_surfel), so that the footprints its warps gather at the same time overlap in L1 as in a plain
// launch; the block waits for its slowest warp before the next item.
__device__ __forceinline__ void batch_square_loop(const PlanParams* __restrict__ plans, const WorkItem* __restrict__ items,
                                                  int n_items, int* __restrict__ counter, int iters, int max_frames,
                                                  PlanParams* spp, float* sdyn, int* s_item) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int group_words = group_scratch_words(max_frames);
    float* wref = sdyn + warp * kBatchGroups * group_words;
    PlanParams* pp = &spp[0];
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = *s_item;
        if (it >= n_items) break;
        const WorkItem w = items[it];
        if (w.plan != cur) {
            const int* src = reinterpret_cast<const int*>(plans + w.plan);
            int* dst = reinterpret_cast<int*>(pp);
            const int n = plan_words(__ldg(&plans[w.plan].F));
            for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = __ldg(src + i);
            __syncthreads();
            cur = w.plan;
        }
        auto run = [&](auto p_tag, auto dt_tag) {
            constexpr int P = decltype(p_tag)::value, DT = decltype(dt_tag)::value, G = batch_lanes(0, P);
            const int s = square_surfel(pp->TX, pp->TY, kBatchBlock / G, w.first, threadIdx.x / G);
            gn_surfel<P, G, DT, false, 4, 0, false, 4>(pp, s < 0 ? pp->S : s, lane % G, iters, kModeSolve,
                                                        wref + (lane / G) * group_words);
        };
        auto by_patch = [&](auto dt_tag) {
            switch (pp->P) {
                case 4: run(std::integral_constant<int, 4>{}, dt_tag); break;
                case 8: run(std::integral_constant<int, 8>{}, dt_tag); break;
                case 16: run(std::integral_constant<int, 16>{}, dt_tag); break;
                default: break;
            }
        };
        switch (pp->dtype) {
            case SGN_F32: by_patch(std::integral_constant<int, SGN_F32>{}); break;
            case SGN_F16: by_patch(std::integral_constant<int, SGN_F16>{}); break;
            case SGN_BF16: by_patch(std::integral_constant<int, SGN_BF16>{}); break;
            case SGN_F16G: by_patch(std::integral_constant<int, SGN_F16G>{}); break;
            case SGN_BF16G: by_patch(std::integral_constant<int, SGN_BF16G>{}); break;
            default: break;
        }
        __syncthreads();  // every warp is done with this item (and with *s_item) before the next
    }
}

// Occupancy and launch of a batch kernel (the counter is reset on the stream first).
template <typename Kernel>
inline int batch_blocks_per_sm_of(Kernel kernel, LaunchAttrs& attrs, int block_threads, int max_frames) {
    if (max_frames < 1 || max_frames > kMaxFrames) return 0;
    if (configure_launch(kernel, attrs, batch_scratch_bytes(kMaxFrames), batch_scratch_bytes(max_frames), 2) != cudaSuccess)
        return 0;
    int n = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block_threads, batch_scratch_bytes(max_frames)) ==
                   cudaSuccess
               ? n
               : 0;
}

template <typename Kernel>
inline int launch_batch_kernel(Kernel kernel, LaunchAttrs& attrs, const PlanParams* d_plans, const WorkItem* d_items,
                               int n_items, int* d_counter, int iters, int grid, int block_threads, int max_frames,
                               cudaStream_t st) {
    if (block_threads != kBatchBlock || max_frames < 1 || max_frames > kMaxFrames) return int(cudaErrorInvalidConfiguration);
    const size_t smem = batch_scratch_bytes(max_frames);
    cudaError_t e = configure_launch(kernel, attrs, batch_scratch_bytes(kMaxFrames), int(smem), 2);
    if (e != cudaSuccess) return int(e);
    e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return int(e);
    kernel<<<grid, block_threads, smem, st>>>(d_plans, d_items, n_items, d_counter, iters, max_frames);
    return int(cudaGetLastError());
}

}  // namespace sgn
