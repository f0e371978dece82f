// Integrator variants for three coupled Hodgkin-Huxley neurons (paper Eq. 6-11).
#include "ff_device.cuh"

namespace ff {
cudaError_t launch_integrate_hh3(int method, bool kahan, bool pp, const IntegrateArgs& a,
                                 const LaunchShape& shape, cudaStream_t stream) {
    return launch_variants<HH3>(method, kahan, pp, a, shape, stream);
}
}  // namespace ff
