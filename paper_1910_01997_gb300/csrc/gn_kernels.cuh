// Plain (one keyframe, one launch) Gauss-Newton kernel and its launcher, instantiated per
// texel dtype by gn_f32.cu / gn_f16.cu / gn_bf16.cu.
#pragma once

#include "gn_impl.cuh"

namespace sgn {

// Copy the plan parameters into shared memory (all threads of the block).
__device__ __forceinline__ void load_plan(PlanParams* dst, const PlanParams* src) {
    static_assert(sizeof(PlanParams) % 4 == 0, "plan params are copied as words");
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < int(sizeof(PlanParams) / 4); i += blockDim.x) d[i] = s[i];
}

template <int P, int G, int DT>
__global__ void __launch_bounds__(256) k_gn(const __grid_constant__ PlanParams pp, int iters, int mode) {
    __shared__ PlanParams spp;
    load_plan(&spp, &pp);
    __syncthreads();
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    gn_surfel<P, G, DT>(&spp, gtid / G, threadIdx.x % G, iters, mode);
}

template <int DT>
int launch_gn_dtype(const PlanParams& pp, int iters, int mode, int G, int block, void* stream) {
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long threads = (long long)pp.S * G;
    const int grid = int((threads + block - 1) / block);
    if (grid == 0) return cudaSuccess;
#define SGN_GN_CASE(PP, GG)                                                          \
    if (pp.P == PP && G == GG) {                                                    \
        k_gn<PP, GG, DT><<<grid, block, 0, st>>>(pp, iters, mode);                   \
        return int(cudaGetLastError());                                             \
    }
    SGN_GN_CASE(4, 8)
    SGN_GN_CASE(4, 16)
    SGN_GN_CASE(8, 8)
    SGN_GN_CASE(8, 16)
    SGN_GN_CASE(8, 32)
    SGN_GN_CASE(16, 32)
#undef SGN_GN_CASE
    return int(cudaErrorInvalidConfiguration);
}

}  // namespace sgn
