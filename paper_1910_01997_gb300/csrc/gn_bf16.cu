// Gauss-Newton kernels with SGN_BF16 frame texels.
#include "gn_kernels.cuh"

namespace sgn {
int launch_gn_bf16(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap) {
    return launch_gn_dtype<SGN_BF16>(pp, iters, mode, G, block, stream, tmap);
}
}  // namespace sgn
