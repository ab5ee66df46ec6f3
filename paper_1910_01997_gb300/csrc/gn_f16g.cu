// Gauss-Newton kernels with SGN_F16G frame texels (FP16 gradients and FP32 intensities).
#include "gn_kernels.cuh"

namespace sgn {
int launch_gn_f16g(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap) {
    return launch_gn_dtype<SGN_F16G>(pp, iters, mode, G, block, stream, tmap);
}
}  // namespace sgn
