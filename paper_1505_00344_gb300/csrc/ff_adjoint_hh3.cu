// ff_adjoint_hh3.cu -- adjoint kernels of the three HH neurons, instantiated in a unit of their own
// so the adjoint compiles in parallel.
#include "ff_adjoint_impl.cuh"

namespace ff {

cudaError_t launch_adjoint_hh3(int method, bool pp, int m, const AdjointArgs& a, int block, int num_sms,
                               cudaStream_t s, int64_t* rows) {
    return launch_r<HH3>(method, pp, m, a, block, num_sms, s, rows);
}

cudaError_t launch_batch_adjoint_hh3(int method, bool pp, int m, const BatchAdjointArgs& b, int num_sms,
                                     cudaStream_t s) {
    return launch_batch_r<HH3>(method, pp, m, b, num_sms, s);
}

}  // namespace ff
