// ff_adjoint.cu -- discrete adjoint of the RK4 / Euler integrator (not part of
// the paper): gradients of a loss of the final states with respect to the
// initial states and the parameters, by reverse sweeps over checkpointed chunks.
//
// One thread per particle walks the chunks in reverse with the adjoint state
// lambda = dL/dx in registers.  A chunk of L <= M*M steps is recomputed from its
// checkpoint twice (once when L <= M): once to place sub-checkpoints every M steps (local memory),
// then per sub-segment (in reverse) to put its <= M states in a shared-memory
// column per thread, which the reverse RK4 steps consume from
// last to first.  The 15-dimensional system is recomputed once per chunk into a
// per-thread scratch area in global memory instead (ff_adjoint_hh3.cu).  Parameter gradients are
// summed per particle in FP32 within a chunk, added to FP64 per chunk, and
// reduced over particles through per-block FP64 partials in fixed order.
//
// This unit holds the dispatch over systems and the fixed-order reductions; the
// kernels themselves are instantiated per family in ff_adjoint_lorenz.cu,
// ff_adjoint_hh3.cu, ff_adjoint_small.cu and ff_adjoint_linear.cu (device code in
// ff_adjoint_impl.cuh).
#include <cstdint>
#include <cuda_runtime.h>

#include "ff.h"
#include "ff_adjoint.h"

namespace ff {

// dp[m * np_stride + q] = sum over rows [row0[m], row0[m + 1]) of partial[row][q], in row order.
__global__ void reduce_member_rows_kernel(const double* partial, const int* row0, int n_members, int np,
                                          int np_stride, double* dp) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n_members * np) return;
    const int m = idx / np, q = idx % np;
    double s = 0.0;
    for (int r = row0[m]; r < row0[m + 1]; ++r) s += partial[(int64_t)r * np_stride + q];
    dp[(int64_t)m * np_stride + q] = s;
}

// Sum of the per-block (or per-warp) partials, in a fixed order.
__global__ void reduce_partials_kernel(const double* partial, int64_t rows, int np, int np_stride, double* out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= np) return;
    double s = 0.0;
    for (int64_t r = 0; r < rows; ++r) s += partial[r * np_stride + q];
    out[q] = s;
}

bool adjoint_supported(int rhs_id) {
    return rhs_id == FF_RHS_LORENZ || rhs_id == FF_RHS_WILSON_COWAN || rhs_id == FF_RHS_HARMONIC ||
           rhs_id == FF_RHS_LINEAR || rhs_id == FF_RHS_HH3;
}

int adjoint_sub_steps(int64_t checkpoint_every) {
    // a chunk of up to 16 steps is one sub-segment (one recomputation); longer chunks take
    // sub-checkpoints every M steps with M * M >= the chunk (two recomputations)
    if (checkpoint_every <= 4) return 4;
    if (checkpoint_every <= 8) return 8;
    if (checkpoint_every <= 16) return 16;
    if (checkpoint_every <= 64) return 8;
    return 16;
}

int64_t adjoint_partial_rows(int num_sms) { return (int64_t)num_sms * 8 * 8; }

int64_t adjoint_scratch_threads(int rhs_id, int method, bool pp, int num_sms, bool batched) {
    return rhs_id == FF_RHS_HH3 ? adjoint_scratch_threads_hh3(method, pp, num_sms, batched) : 0;
}

cudaError_t launch_adjoint(int rhs_id, int method, bool pp, int m, const AdjointArgs& a, int num_sms,
                           cudaStream_t s, double* dL_dp_dev, int n_params_kernel) {
    const int block = 128;
    int64_t rows = 0;
    cudaError_t e;
    switch (rhs_id) {
    case FF_RHS_LORENZ: e = launch_adjoint_lorenz(method, pp, m, a, block, num_sms, s, &rows); break;
    case FF_RHS_HH3: e = launch_adjoint_hh3(method, pp, m, a, block, num_sms, s, &rows); break;
    case FF_RHS_LINEAR: e = launch_adjoint_linear(method, pp, m, a, block, num_sms, s, &rows); break;
    case FF_RHS_WILSON_COWAN:
    case FF_RHS_HARMONIC: e = launch_adjoint_small(rhs_id, method, pp, m, a, block, num_sms, s, &rows); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    reduce_partials_kernel<<<(n_params_kernel + 63) / 64, 64, 0, s>>>(a.partial, rows, n_params_kernel, a.np_stride,
                                                                       dL_dp_dev);
    return cudaGetLastError();
}

cudaError_t launch_batch_adjoint(int rhs_id, int method, bool pp, int m, const BatchAdjointArgs& b,
                                 const int* row0_dev, int n_members, int n_params_kernel, int num_sms,
                                 cudaStream_t s, double* dp_dev) {
    cudaError_t e;
    switch (rhs_id) {
    case FF_RHS_LORENZ: e = launch_batch_adjoint_lorenz(method, pp, m, b, num_sms, s); break;
    case FF_RHS_HH3: e = launch_batch_adjoint_hh3(method, pp, m, b, num_sms, s); break;
    case FF_RHS_LINEAR: e = launch_batch_adjoint_linear(method, pp, m, b, num_sms, s); break;
    case FF_RHS_WILSON_COWAN:
    case FF_RHS_HARMONIC: e = launch_batch_adjoint_small(rhs_id, method, pp, m, b, num_sms, s); break;
    default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int items = n_members * n_params_kernel;
    if (items > 0)
        reduce_member_rows_kernel<<<(items + 127) / 128, 128, 0, s>>>(b.partial, row0_dev, n_members,
                                                                      n_params_kernel, b.np_stride, dp_dev);
    return cudaGetLastError();
}

}  // namespace ff
