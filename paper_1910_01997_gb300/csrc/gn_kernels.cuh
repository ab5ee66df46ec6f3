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

// Minimum resident 256-thread blocks per SM (register budget 85 / 128 / 255 per thread) by pixels
// per lane: with 4800 surfels of 8x8 pixels (a 640x480 keyframe) at 16 or 8 lanes per surfel every
// surfel is resident in a single wave on 152 SMs.
constexpr int gn_min_blocks(int P, int G) { return P * P / G <= 2 ? 3 : (P * P / G == 4 ? 2 : 1); }
constexpr int kRefStride = kMaxFrames * kRefWords + 1;  // odd stride: groups of a warp use distinct banks

template <int P, int G, int DT>
__global__ void __launch_bounds__(256, gn_min_blocks(P, G)) k_gn(const __grid_constant__ PlanParams pp, int iters, int mode) {
    __shared__ PlanParams spp;
    __shared__ float sref[256 / G][kRefStride];
    load_plan(&spp, &pp);
    __syncthreads();
    const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
    gn_surfel<P, G, DT>(&spp, gtid / G, threadIdx.x % G, iters, mode, sref[threadIdx.x / G]);
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
