// ff_adjoint_lorenz.cu -- adjoint kernels of Lorenz, instantiated in a unit of their own
// so the adjoint compiles in parallel.
#include "ff_adjoint_impl.cuh"

namespace ff {

cudaError_t launch_adjoint_lorenz(int method, bool pp, int m, const AdjointArgs& a, int block, int num_sms,
                                  cudaStream_t s, int64_t* rows) {
    // RK4: the packed-pair sweep; Euler: the scalar one
    return method == FF_RK4 ? launch_lorenz_x2(pp, m, a, num_sms, s, rows)
                            : launch_r<Lorenz>(method, pp, m, a, block, num_sms, s, rows);
}

cudaError_t launch_batch_adjoint_lorenz(int method, bool pp, int m, const BatchAdjointArgs& b, int num_sms,
                                        cudaStream_t s) {
    return launch_batch_r<Lorenz>(method, pp, m, b, num_sms, s);
}

}  // namespace ff
