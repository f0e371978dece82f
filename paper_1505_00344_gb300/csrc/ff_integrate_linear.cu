// Integrator variants for the linear test systems (dx/dt = A x, harmonic oscillator).
#include "ff_device.cuh"

namespace ff {
cudaError_t launch_integrate_linear(int rhs_id, int method, bool kahan, bool pp,
                                    const IntegrateArgs& a, const LaunchShape& shape,
                                    cudaStream_t stream) {
    if (rhs_id == FF_RHS_HARMONIC) return launch_variants<Harmonic>(method, kahan, pp, a, shape, stream);
    return launch_variants<Linear>(method, kahan, pp, a, shape, stream);
}
}  // namespace ff
