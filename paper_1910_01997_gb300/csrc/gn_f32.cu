// Gauss-Newton kernels with SGN_F32 frame texels, and the FP64 solve diagnostic.
#include "gn_kernels.cuh"

namespace sgn {
int launch_gn_f32(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap) {
    return launch_gn_dtype<SGN_F32>(pp, iters, mode, G, block, stream, tmap);
}
}  // namespace sgn

// ------------------------------------------------------------------------------ diagnostics

namespace {
// One damped system per group of 16 lanes, solved by the same device function as the
// Gauss-Newton kernels' FP64 route.
__global__ void __launch_bounds__(256) k_fp64_solve(const float* H6, const float* g3, double lambda, int n,
                                                    float* delta, int* pd) {
    const int sys = (blockIdx.x * blockDim.x + threadIdx.x) / 16, lg = threadIdx.x % 16;
    const bool active = sys < n;
    float H[6] = {1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 1.0f}, g[3] = {0.0f, 0.0f, 0.0f}, d[3];
    if (active) {
        for (int k = 0; k < 6; ++k) H[k] = H6[6 * sys + k];
        for (int k = 0; k < 3; ++k) g[k] = g3[3 * sys + k];
    }
    const bool ok = sgn::solve_f64_route<16>(H, g, lambda, active, lg, d);
    if (active && lg == 0) {
        for (int k = 0; k < 3; ++k) delta[3 * sys + k] = d[k];
        pd[sys] = ok ? 1 : 0;
    }
}
}  // namespace

extern "C" sgn_status sgn_check_fp64_solve(const float* H6, const float* g3, double lambda, int n, float* delta,
                                           int32_t* pd, void* stream) {
    if (n < 0 || (n > 0 && (!H6 || !g3 || !delta || !pd)) || !(lambda >= 0.0))
        return sgn::record_error(SGN_ERR_INVALID_ARGUMENT, "NULL array, n < 0 or lambda not >= 0");
    if (n == 0) return SGN_OK;
    const long long threads = 16LL * n;
    k_fp64_solve<<<unsigned((threads + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(H6, g3, lambda, n, delta, pd);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sgn::record_error(SGN_ERR_CUDA, cudaGetErrorString(e));
    sgn::count_launch();
    return SGN_OK;
}
