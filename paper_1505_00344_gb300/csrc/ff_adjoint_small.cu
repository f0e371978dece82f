// ff_adjoint_small.cu -- adjoint kernels of Wilson-Cowan and the harmonic oscillator, instantiated in a unit of their own
// so the adjoint compiles in parallel.
#include "ff_adjoint_impl.cuh"

namespace ff {

cudaError_t launch_adjoint_small(int rhs_id, int method, bool pp, int m, const AdjointArgs& a, int block,
                                 int num_sms, cudaStream_t s, int64_t* rows) {
    switch (rhs_id) {
    case FF_RHS_WILSON_COWAN: return launch_r<WilsonCowan>(method, pp, m, a, block, num_sms, s, rows);
    case FF_RHS_HARMONIC: return launch_r<Harmonic>(method, pp, m, a, block, num_sms, s, rows);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_adjoint_small(int rhs_id, int method, bool pp, int m, const BatchAdjointArgs& b,
                                       int num_sms, cudaStream_t s) {
    switch (rhs_id) {
    case FF_RHS_WILSON_COWAN: return launch_batch_r<WilsonCowan>(method, pp, m, b, num_sms, s);
    case FF_RHS_HARMONIC: return launch_batch_r<Harmonic>(method, pp, m, b, num_sms, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ff
