// Gauss-Newton kernels with SGN_F32 frame texels, and the FP64 reciprocal diagnostic.
#include "gn_kernels.cuh"

namespace sgn {
int launch_gn_f32(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap) {
    return launch_gn_dtype<SGN_F32>(pp, iters, mode, G, block, stream, tmap);
}
}  // namespace sgn

// ------------------------------------------------------------------------------ diagnostics

namespace {
__global__ void __launch_bounds__(256) k_fp64_reciprocal(const double* x, double* r, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = sgn::rcp64(x[i]);
}
}  // namespace

extern "C" sgn_status sgn_check_fp64_reciprocal(const double* x, double* r, int n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !r))) return sgn::record_error(SGN_ERR_INVALID_ARGUMENT, "x/r NULL or n < 0");
    if (n == 0) return SGN_OK;
    k_fp64_reciprocal<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, r, n);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sgn::record_error(SGN_ERR_CUDA, cudaGetErrorString(e));
    sgn::count_launch();
    return SGN_OK;
}
