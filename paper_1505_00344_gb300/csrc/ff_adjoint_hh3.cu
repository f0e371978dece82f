// ff_adjoint_hh3.cu -- adjoint kernels of the three HH neurons (the staged sweep),
// instantiated in a unit of their own so the adjoint compiles in parallel.
#include "ff_adjoint_impl.cuh"

namespace ff {

cudaError_t launch_adjoint_hh3(int method, bool pp, int /*m*/, const AdjointArgs& a, int /*block*/, int num_sms,
                               cudaStream_t s, int64_t* rows) {
    return launch_staged<HH3>(method, pp, a, num_sms, s, rows);
}

cudaError_t launch_batch_adjoint_hh3(int method, bool pp, int /*m*/, const BatchAdjointArgs& b, int num_sms,
                                     cudaStream_t s) {
    return launch_batch_staged<HH3>(method, pp, b, num_sms, s);
}

int64_t adjoint_scratch_threads_hh3(int method, bool pp, int num_sms, bool batched) {
    return batched ? staged_threads_for<HH3, true>(method, pp, num_sms)
                   : staged_threads_for<HH3, false>(method, pp, num_sms);
}

}  // namespace ff
