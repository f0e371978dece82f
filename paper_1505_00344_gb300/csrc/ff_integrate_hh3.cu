// Integrator variants for three coupled Hodgkin-Huxley neurons (paper Eq. 6-11).
#include "ff_device.cuh"

namespace ff {

namespace {

// Two particles per thread, all three neurons packed across the pair (hh3_rk4_x2_item).
template <bool PP, bool TAPE>
__global__ void __launch_bounds__(HH3::MAX_BLOCK / 2, 3) hh3_rk4_x2_kernel(const __grid_constant__ IntegrateArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = warp_major_first(blockIdx.x, gridDim.x); t < a.n_vec; t += stride)
        hh3_rk4_x2_item<PP, TAPE>(a, t, (int)a.n_steps);
}

}  // namespace

cudaError_t launch_integrate_hh3(int method, bool kahan, bool pp, const IntegrateArgs& a,
                                 const LaunchShape& shape, cudaStream_t stream) {
    if (shape.ppt == 2) {
        // pairs when they fill one wave of the pair kernel (3 blocks of 128 per SM); a smaller
        // ensemble keeps more threads at one particle each (the same bits either way)
        const bool fills = a.n_vec >= (int64_t)shape.num_sms * 3 * (HH3::MAX_BLOCK / 2);
        if (method == FF_RK4 && !kahan && !a.reset && fills) {
            if (a.ckpt)
                return pp ? persistent_launch(hh3_rk4_x2_kernel<true, true>, a, shape, stream)
                          : persistent_launch(hh3_rk4_x2_kernel<false, true>, a, shape, stream);
            return pp ? persistent_launch(hh3_rk4_x2_kernel<true, false>, a, shape, stream)
                      : persistent_launch(hh3_rk4_x2_kernel<false, false>, a, shape, stream);
        }
        // Euler, the compensated update, particle reset and small ensembles: one particle per thread
        IntegrateArgs a1 = a;
        LaunchShape s1 = shape;
        a1.n_vec = a.n_vec * 2;
        s1.ppt = 1;
        return launch_variants<HH3>(method, kahan, pp, a1, s1, stream);
    }
    return launch_variants<HH3>(method, kahan, pp, a, shape, stream);
}

}  // namespace ff
