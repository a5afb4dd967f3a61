// Adjoint of the moment rasterizer (filled in by the backward implementation).
#include "common.cuh"

namespace mb {
int launch_backward(const Params&, const ViewTable&, const Layout&, char*, const mb3dgs_gaussians&, const float*,
                    const float*, const mb3dgs_gaussian_grads&, cudaStream_t) {
    return MB3DGS_ERR_UNSUPPORTED;
}
}  // namespace mb
