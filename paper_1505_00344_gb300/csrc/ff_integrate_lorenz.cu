// Integrator variants for the Lorenz system (paper Eq. 3-5).
#include "ff_device.cuh"

namespace ff {

// Whether the group-uniform packed kernel runs for these arguments (the only
// kernel with the fused splat epilogue).
bool lorenz_uniform_packed(int method, bool kahan, bool pp, const IntegrateArgs& a, const LaunchShape& shape) {
    if (method != FF_RK4 || kahan || a.reset || (shape.ppt != 2 && shape.ppt != 4)) return false;
    for (int g = 0; g < a.n_groups; ++g)
        if (a.gstart[g] % shape.ppt != 0) return false;
    return !pp || a.pidx == 1;
}

cudaError_t launch_integrate_lorenz_splat(bool pp, const IntegrateArgs& a, const LaunchShape& shape,
                                          cudaStream_t stream) {
    if (shape.ppt == 2)
        return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 1, true>, a, shape, stream)
                  : uniform_launch(lorenz_rk4_x2u_kernel<false, 1, true>, a, shape, stream);
    return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 2, true>, a, shape, stream)
              : uniform_launch(lorenz_rk4_x2u_kernel<false, 2, true>, a, shape, stream);
}

cudaError_t launch_integrate_lorenz(int method, bool kahan, bool pp, const IntegrateArgs& a,
                                    const LaunchShape& shape, cudaStream_t stream) {
    // plain RK4 at 2 or 4 particles per thread runs as packed f32x2 pairs (without resets)
    if (method == FF_RK4 && !kahan && !a.reset && (shape.ppt == 2 || shape.ppt == 4)) {
        bool aligned = true;
        for (int g = 0; g < a.n_groups; ++g) aligned = aligned && (a.gstart[g] % shape.ppt == 0);
        if (aligned && (!pp || a.pidx == 1)) {
            if (shape.ppt == 2)
                return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 1>, a, shape, stream)
                          : uniform_launch(lorenz_rk4_x2u_kernel<false, 1>, a, shape, stream);
            return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 2>, a, shape, stream)
                      : uniform_launch(lorenz_rk4_x2u_kernel<false, 2>, a, shape, stream);
        }
        if (shape.ppt == 2)
            return pp ? persistent_launch(lorenz_rk4_x2_kernel<true, 1>, a, shape, stream)
                      : persistent_launch(lorenz_rk4_x2_kernel<false, 1>, a, shape, stream);
        return pp ? persistent_launch(lorenz_rk4_x2_kernel<true, 2>, a, shape, stream)
                  : persistent_launch(lorenz_rk4_x2_kernel<false, 2>, a, shape, stream);
    }
    return launch_variants<Lorenz>(method, kahan, pp, a, shape, stream);
}

}  // namespace ff
