// Integrator variants for the Lorenz system (paper Eq. 3-5).
#include "ff_device.cuh"

namespace ff {

// Deal the persistent grid's blocks out to the groups in proportion to their
// sizes (at least one block per group) and launch the group-uniform kernel.
template <class Kernel>
static cudaError_t uniform_launch(Kernel kernel, const IntegrateArgs& a0, const LaunchShape& s0,
                                  cudaStream_t stream) {
    LaunchShape s = s0;
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, kernel);
    if (e != cudaSuccess) return e;
    if (s.block > attr.maxThreadsPerBlock) s.block = attr.maxThreadsPerBlock / 32 * 32;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, s.block, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = (s.blocks_per_sm > 0 && s.blocks_per_sm < occ) ? s.blocks_per_sm : occ;
    const int64_t total = (int64_t)per_sm * s.num_sms;
    IntegrateArgs a = a0;
    const int ppt = s.ppt;
    int64_t items_all = 0;
    for (int g = 0; g < a.n_groups; ++g) items_all += (a.gend[g] - a.gstart[g]) / ppt;
    int next = 0;
    for (int g = 0; g < a.n_groups; ++g) {
        const int64_t items = (a.gend[g] - a.gstart[g]) / ppt;
        int64_t nb = items_all > 0 ? (total * items + items_all / 2) / items_all : 1;
        const int64_t need = (items + s.block - 1) / s.block;
        if (nb > need) nb = need;
        if (nb < 1) nb = 1;
        a.gblk[g] = next;
        next += (int)nb;
    }
    a.gblk[a.n_groups] = next;
    kernel<<<next, s.block, 0, stream>>>(a);
    return cudaGetLastError();
}

// Whether the group-uniform packed kernel runs for these arguments (the only
// kernel with the fused splat epilogue).
bool lorenz_uniform_packed(int method, bool kahan, bool pp, const IntegrateArgs& a, const LaunchShape& shape) {
    if (method != FF_RK4 || kahan || a.reset || (shape.ppt != 2 && shape.ppt != 4)) return false;
    for (int g = 0; g < a.n_groups; ++g)
        if (a.gstart[g] % shape.ppt != 0) return false;
    return !pp || a.pidx == 1;
}

cudaError_t launch_integrate_lorenz_splat(bool pp, const IntegrateArgs& a, const LaunchShape& shape,
                                          cudaStream_t stream) {
    if (shape.ppt == 2)
        return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 1, true>, a, shape, stream)
                  : uniform_launch(lorenz_rk4_x2u_kernel<false, 1, true>, a, shape, stream);
    return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 2, true>, a, shape, stream)
              : uniform_launch(lorenz_rk4_x2u_kernel<false, 2, true>, a, shape, stream);
}

cudaError_t launch_integrate_lorenz(int method, bool kahan, bool pp, const IntegrateArgs& a,
                                    const LaunchShape& shape, cudaStream_t stream) {
    // plain RK4 at 2 or 4 particles per thread runs as packed f32x2 pairs (without resets)
    if (method == FF_RK4 && !kahan && !a.reset && (shape.ppt == 2 || shape.ppt == 4)) {
        bool aligned = true;
        for (int g = 0; g < a.n_groups; ++g) aligned = aligned && (a.gstart[g] % shape.ppt == 0);
        if (aligned && (!pp || a.pidx == 1)) {
            if (shape.ppt == 2)
                return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 1>, a, shape, stream)
                          : uniform_launch(lorenz_rk4_x2u_kernel<false, 1>, a, shape, stream);
            return pp ? uniform_launch(lorenz_rk4_x2u_kernel<true, 2>, a, shape, stream)
                      : uniform_launch(lorenz_rk4_x2u_kernel<false, 2>, a, shape, stream);
        }
        if (shape.ppt == 2)
            return pp ? persistent_launch(lorenz_rk4_x2_kernel<true, 1>, a, shape, stream)
                      : persistent_launch(lorenz_rk4_x2_kernel<false, 1>, a, shape, stream);
        return pp ? persistent_launch(lorenz_rk4_x2_kernel<true, 2>, a, shape, stream)
                  : persistent_launch(lorenz_rk4_x2_kernel<false, 2>, a, shape, stream);
    }
    return launch_variants<Lorenz>(method, kahan, pp, a, shape, stream);
}

}  // namespace ff
