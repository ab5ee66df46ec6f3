// Gauss-Newton kernels with SGN_F16 frame texels.
#include "gn_kernels.cuh"

namespace sgn {
int launch_gn_f16(const PlanParams& pp, int iters, int mode, int G, int block, void* stream, const void* tmap) {
    return launch_gn_dtype<SGN_F16>(pp, iters, mode, G, block, stream, tmap);
}
}  // namespace sgn
