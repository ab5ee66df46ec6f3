// Gauss-Newton kernels with SGN_BF16G frame texels (BF16 gradients and FP32 intensities).
#include "gn_kernels.cuh"

namespace sgn {
int launch_gn_bf16g(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap) {
    return launch_gn_dtype<SGN_BF16G>(pp, iters, mode, G, block, stream, tmap);
}
}  // namespace sgn
