// Integrator variants for the Lorenz system (paper Eq. 3-5).
#include "ff_device.cuh"

namespace ff {
cudaError_t launch_integrate_lorenz(int method, bool kahan, bool pp, const IntegrateArgs& a,
                                    const LaunchShape& shape, cudaStream_t stream) {
    // plain RK4 at 2 or 4 particles per thread runs as packed f32x2 pairs
    if (method == FF_RK4 && !kahan && (shape.ppt == 2 || shape.ppt == 4)) {
        if (shape.ppt == 2)
            return pp ? persistent_launch(lorenz_rk4_x2_kernel<true, 1>, a, shape, stream)
                      : persistent_launch(lorenz_rk4_x2_kernel<false, 1>, a, shape, stream);
        return pp ? persistent_launch(lorenz_rk4_x2_kernel<true, 2>, a, shape, stream)
                  : persistent_launch(lorenz_rk4_x2_kernel<false, 2>, a, shape, stream);
    }
    return launch_variants<Lorenz>(method, kahan, pp, a, shape, stream);
}
}  // namespace ff
