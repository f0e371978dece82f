// Integrator variants for the Lorenz system (paper Eq. 3-5).
#include "ff_device.cuh"

namespace ff {
cudaError_t launch_integrate_lorenz(int method, bool kahan, bool pp, const IntegrateArgs& a,
                                    const LaunchShape& shape, cudaStream_t stream) {
    return launch_variants<Lorenz>(method, kahan, pp, a, shape, stream);
}
}  // namespace ff
