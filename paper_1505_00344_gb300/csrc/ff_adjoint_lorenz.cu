// ff_adjoint_lorenz.cu -- adjoint kernels of Lorenz, instantiated in a unit of their own
// so the adjoint compiles in parallel.
#include "ff_adjoint_impl.cuh"

namespace ff {

// The packed-pair sweeps' launcher.  It is defined in this unit rather than in the shared
// header: as a non-template function there it would compile these kernels into every
// adjoint unit.
static cudaError_t launch_lorenz_x2(bool pp, int m, const AdjointArgs& a, int num_sms, cudaStream_t s,
                                    int64_t* rows) {
    // chunks of up to 16 steps are one sub-segment (one recomputation); longer ones take the
    // sweep with 4-step sub-segments that keep their stage points
    if (a.max_chunk > 16) {
        if (a.max_chunk > kLx2sSub * kLx2sMaxSub) return cudaErrorInvalidValue;
        return pp ? launch_lorenz_x2_kernel(adjoint_lorenz_x2s_kernel<true>, a, num_sms, s, rows)
                  : launch_lorenz_x2_kernel(adjoint_lorenz_x2s_kernel<false>, a, num_sms, s, rows);
    }
    switch (m) {
    case 4: return pp ? launch_lorenz_x2_one<true, 4>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 4>(a, num_sms, s, rows);
    case 8: return pp ? launch_lorenz_x2_one<true, 8>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 8>(a, num_sms, s, rows);
    case 16: return pp ? launch_lorenz_x2_one<true, 16>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 16>(a, num_sms, s, rows);
    default: return cudaErrorInvalidValue;
    }
}

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
