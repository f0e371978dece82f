// Integrator variants for the Wilson-Cowan E-I model (paper Eq. 1-2).
#include "ff_device.cuh"

namespace ff {
cudaError_t launch_integrate_wc(int method, bool kahan, bool pp, const IntegrateArgs& a,
                                const LaunchShape& shape, cudaStream_t stream) {
    return launch_variants<WilsonCowan>(method, kahan, pp, a, shape, stream);
}
}  // namespace ff
