// Plain (one keyframe, one launch) Gauss-Newton kernel and its launcher, instantiated per
// texel dtype by gn_f32.cu / gn_f16.cu / gn_bf16.cu.
#pragma once

#include <algorithm>
#include <cstring>

#include "gn_impl.cuh"

namespace sgn {

// Copy the plan parameters into shared memory (all threads of the block): the fields before the
// frame poses and the poses of the frames in use (the unused slots are never read).
__device__ __forceinline__ void load_plan(PlanParams* dst, const PlanParams* src) {
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    const int n = plan_words(src->F);
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = s[i];
}

// Minimum resident 256-thread blocks per SM (register budget 85 / 128 / 255 per thread) by pixels
// per lane: with 4800 surfels of 8x8 pixels (a 640x480 keyframe) at 16 or 8 lanes per surfel every
// surfel is resident in a single wave on 152 SMs.
constexpr int gn_min_blocks(int P, int G) { return P * P / G <= 2 ? 3 : (P * P / G == 4 ? 2 : 1); }

// Dynamic shared memory of a launch: each group's frame scratch (group_scratch_words(F) floats,
// 16-byte aligned), then, when staging, each group's texel boxes (128-byte aligned).
__host__ __device__ constexpr int scratch_bytes(int groups, int F) { return groups * group_scratch_words(F) * 4; }

// This thread's surfel in a plain launch (the block's square of tiles); S when its group has none.
__device__ __forceinline__ int block_surfel(const PlanParams& pp, int G) {
    const int s = square_surfel(pp.TX, pp.TY, blockDim.x / G, blockIdx.x, threadIdx.x / G);
    return s < 0 ? pp.S : s;
}

// BT: most threads per block.  256-thread blocks take a 4 x 4 square of tiles (16 groups of 16 lanes);
// a 512-thread block takes 8 x 4 tiles, the share of one SM at 640x480 (4800 surfels on 152 SMs),
// whose texel footprint per frame is smaller than that of two separate 4 x 4 squares.
template <int P, int G, int DT, bool LMA = false, int BT = 256>
__global__ void __launch_bounds__(BT, BT > 256 ? 1 : gn_min_blocks(P, G)) k_gn(const __grid_constant__ PlanParams pp, int iters, int mode) {
    __shared__ PlanParams spp;
    extern __shared__ float4 sdyn[];
    load_plan(&spp, &pp);
    __syncthreads();
    float* scratch = reinterpret_cast<float*>(sdyn) + (threadIdx.x / G) * group_scratch_words(pp.F);
    gn_surfel<P, G, DT, false, 8, 0, LMA>(&spp, block_surfel(pp, G), threadIdx.x % G, iters, mode, scratch);
}

// Staged variant: every group of G lanes also owns kStageSlots texel boxes (box_stride(P, DT) bytes
// each) and one mbarrier per box.
template <int P, int G, int DT>
__global__ void __launch_bounds__(256, gn_min_blocks(P, G))
    k_gn_staged(const __grid_constant__ PlanParams pp, int iters, int mode, const __grid_constant__ TexMap tmap) {
    __shared__ PlanParams spp;
    __shared__ unsigned long long sbar[256 / G][kStageSlots];
    extern __shared__ float4 sdyn[];
    const int grp = threadIdx.x / G, lg = threadIdx.x % G;
    load_plan(&spp, &pp);
    if (lg == 0)
        for (int k = 0; k < kStageSlots; ++k) mbar_init(smem_addr(&sbar[grp][k]), 1);
    fence_mbar_init();
    __syncthreads();
    unsigned char* dyn = reinterpret_cast<unsigned char*>(sdyn);
    const unsigned boxes0 = (smem_addr(dyn) + scratch_bytes(blockDim.x / G, pp.F) + 127u) & ~127u;
    constexpr unsigned group_bytes = kStageSlots * box_stride(P, DT);
    Stage st;
    st.tmap = &tmap;
    st.slots = boxes0 + grp * group_bytes;
    st.bars = smem_addr(&sbar[grp][0]);
    st.slots_ptr = dyn + (st.slots - smem_addr(dyn));
    st.issued = st.consumed = 0;
    st.broken = false;
    float* scratch = reinterpret_cast<float*>(sdyn) + grp * group_scratch_words(pp.F);
    gn_surfel<P, G, DT, true>(&spp, block_surfel(pp, G), lg, iters, mode, scratch, &st);
}

// Circular surfels: one warp per surfel, DPPL disc pixels per lane in passes of four.
template <int P, int DT, int DPPL>
__global__ void __launch_bounds__(256, 2) k_gn_disc(const __grid_constant__ PlanParams pp, int iters, int mode) {
    __shared__ PlanParams spp;
    extern __shared__ float4 sdyn[];
    load_plan(&spp, &pp);
    __syncthreads();
    float* scratch = reinterpret_cast<float*>(sdyn) + (threadIdx.x / 32) * group_scratch_words(pp.F);
    gn_surfel<P, 32, DT, false, 4, DPPL>(&spp, block_surfel(pp, 32), threadIdx.x % 32, iters, mode, scratch);
}

template <int P, int DT, int DPPL>
int launch_disc(const PlanParams& pp, int iters, int mode, int grid, int block, cudaStream_t st) {
    static LaunchAttrs attrs;
    const int smem = scratch_bytes(block / 32, pp.F);
    const cudaError_t e = configure_launch(k_gn_disc<P, DT, DPPL>, attrs, scratch_bytes(8, kMaxFrames), smem, 2 * 256 / block);
    if (e != cudaSuccess) return int(e);
    k_gn_disc<P, DT, DPPL><<<grid, block, smem, st>>>(pp, iters, mode);
    return int(cudaGetLastError());
}

template <int P, int DT>
int launch_disc_ppl(const PlanParams& pp, int iters, int mode, int grid, int block, cudaStream_t st) {
    if (pp.disc_n <= 2 * 32) return launch_disc<P, DT, 2>(pp, iters, mode, grid, block, st);
    if (pp.disc_n <= 4 * 32) return launch_disc<P, DT, 4>(pp, iters, mode, grid, block, st);
    if (pp.disc_n <= 8 * 32) return launch_disc<P, DT, 8>(pp, iters, mode, grid, block, st);
    if (pp.disc_n <= 16 * 32) return launch_disc<P, DT, 16>(pp, iters, mode, grid, block, st);
    return int(cudaErrorInvalidConfiguration);
}

// Plain launch of one Gauss-Newton kernel instantiation (direct gathers).
template <int P, int G, int DT, bool LMA, int BT>
int launch_plain(const PlanParams& pp, int iters, int mode, int grid, int block, cudaStream_t st) {
    static LaunchAttrs attrs;
    const int smem = scratch_bytes(block / G, pp.F);
    const int blocks = BT > 256 ? 1 : gn_min_blocks(P, G) * 256 / block;
    const cudaError_t e = configure_launch(k_gn<P, G, DT, LMA, BT>, attrs, scratch_bytes(BT / G, kMaxFrames), smem, blocks);
    if (e != cudaSuccess) return int(e);
    k_gn<P, G, DT, LMA, BT><<<grid, block, smem, st>>>(pp, iters, mode);
    return int(cudaGetLastError());
}

template <int P, int G, int DT>
int launch_one(const PlanParams& pp, int iters, int mode, int grid, int block, cudaStream_t st, const void* tmap) {
    if (pp.lm_adaptive) return launch_plain<P, G, DT, true, 256>(pp, iters, mode, grid, block, st);  // Marquardt schedule
    if (!tmap && block > 256) {
        if constexpr (P * P / G == 4) return launch_plain<P, G, DT, false, 512>(pp, iters, mode, grid, block, st);
        return int(cudaErrorInvalidConfiguration);
    }
    if (!tmap) return launch_plain<P, G, DT, false, 256>(pp, iters, mode, grid, block, st);
    // staged: boxes of the block's groups after the scratch, plus slack to align them to 128 bytes
    static LaunchAttrs attrs;
    const int boxes = kStageSlots * box_stride(P, DT);
    const int smem = scratch_bytes(block / G, pp.F) + (block / G) * boxes + 128;
    const cudaError_t e = configure_launch(k_gn_staged<P, G, DT>, attrs, scratch_bytes(256 / G, kMaxFrames) + (256 / G) * boxes + 128,
                                           smem, gn_min_blocks(P, G) * 256 / block);
    if (e != cudaSuccess) return int(e);
    TexMap m;
    memcpy(&m, tmap, sizeof m);
    k_gn_staged<P, G, DT><<<grid, block, smem, st>>>(pp, iters, mode, m);
    return int(cudaGetLastError());
}

template <int DT>
int launch_gn_dtype(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap) {
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (block > 512 || block % G || (block > 256 && (block != 512 || tmap || pp.lm_adaptive || pp.disc_n > 0)))
        return int(cudaErrorInvalidConfiguration);
    const int grid = pp.S > 0 ? square_blocks(pp.TX, pp.TY, block / G) : 0;
    if (grid == 0) return cudaSuccess;
    if (pp.disc_n > 0) {  // circular surfels: 32 lanes per surfel, no staging
        if (G != 32) return int(cudaErrorInvalidConfiguration);
        switch (pp.P) {
            case 4: return launch_disc_ppl<4, DT>(pp, iters, mode, grid, block, st);
            case 8: return launch_disc_ppl<8, DT>(pp, iters, mode, grid, block, st);
            case 16: return launch_disc_ppl<16, DT>(pp, iters, mode, grid, block, st);
            default: return int(cudaErrorInvalidConfiguration);
        }
    }
#define SGN_GN_CASE(PP, GG) \
    if (pp.P == PP && G == GG) return launch_one<PP, GG, DT>(pp, iters, mode, grid, block, st, tmap);
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
