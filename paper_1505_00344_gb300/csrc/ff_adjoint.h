// ff_adjoint.h -- argument blocks and launcher of the discrete adjoint.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ff.h"

namespace ff {

// One checkpointed chunk of a taped run: n_steps steps from checkpoint `ckpt`
// with parameters p (kernel layout) and the groups' signed steps gh.
struct AdjChunk {
    int n_steps;
    int ckpt;
    float p[FF_MAX_PARAMS];
    float gh[FF_MAX_GROUPS];
};

struct AdjointArgs {
    const float* ckpt;       // checkpoints, slot c at ckpt + c * dim * pitch (SoA planes)
    const AdjChunk* chunks;  // device table, in time order
    int n_chunks;
    int dim;
    const float* lam_in;     // dL/dx(T), SoA [dim][n], contiguous
    float* lam_out;          // dL/dx(0), same layout (may alias lam_in)
    const float* pparam;     // per-particle parameter values (PP only)
    int pidx;
    int np_stride;           // doubles per partial row
    double* partial;         // per-block (or per-warp) FP64 partial sums of dL/dp
    int64_t max_blocks;      // rows available in `partial` / warps per block
    int64_t n;               // particles
    int64_t pitch;           // floats between checkpoint planes
    int n_groups;
    int max_chunk;           // steps of the longest chunk (the tape's checkpoint spacing)
    int64_t gstart[FF_MAX_GROUPS];
    float* scratch;           // HH x 3 sweep: one chunk of stage points per thread (a neuron of two particles)
    int64_t scratch_threads;  // threads the scratch has room for (see adjoint_scratch_floats_per_step)
};

// Batched adjoint: work tiles of consecutive particles of one member (one
// particle per thread); the parameter gradient of tile t goes to row t of
// `partial`, and rows [row0[m], row0[m + 1]) belong to member m.
struct AdjTile {
    int sys;
    int pad_;
    int64_t first;
    int64_t count;
};

struct BatchAdjointArgs {
    const AdjointArgs* sys;  // per member (its partial / max_blocks / scratch fields unused)
    const AdjTile* tiles;
    int n_tiles;
    int np_stride;           // doubles per partial row
    double* partial;         // n_tiles rows
    float* scratch;          // HH x 3 sweep: one chunk of stage points per thread (as AdjointArgs)
    int64_t scratch_threads;
};

bool adjoint_supported(int rhs_id);
int adjoint_sub_steps(int64_t checkpoint_every);  // M >= K up to 16, else M * M >= K (K at most 256)
int64_t adjoint_partial_rows(int num_sms);
// Threads of the HH x 3 sweep (standalone or batched): each needs a scratch area of
// (largest chunk) x adjoint_scratch_floats_per_step floats; 0 for the systems whose
// sweeps keep their states on chip.
int64_t adjoint_scratch_threads(int rhs_id, int method, bool pp, int num_sms, bool batched);
int64_t adjoint_scratch_threads_hh3(int method, bool pp, int num_sms, bool batched);
cudaError_t launch_adjoint(int rhs_id, int method, bool pp, int m, const AdjointArgs& a, int num_sms,
                           cudaStream_t s, double* dL_dp_dev, int n_params_kernel);
// Scratch floats per thread and step of the HH x 3 sweep (a thread holds one neuron of two
// particles): RK4 keeps the four stage points (4 x 5 f32x2), Euler the state (5 f32x2).
inline int adjoint_scratch_floats_per_step(int rhs_id, int method) {
    return rhs_id == FF_RHS_HH3 ? (method == FF_RK4 ? 40 : 10) : 0;
}
constexpr int kAdjTile = 128;    // particles per batched-adjoint tile = threads per block
constexpr int kAdjTileHH3 = 80;  // HH x 3: 128 threads, three lanes per pair of particles (20 per warp)
inline int adjoint_tile_particles(int rhs_id) { return rhs_id == FF_RHS_HH3 ? kAdjTileHH3 : kAdjTile; }

// Per-family launchers (ff_adjoint_lorenz.cu, ff_adjoint_hh3.cu, ff_adjoint_small.cu,
// ff_adjoint_linear.cu): the sweep
// kernel only; `rows` receives the number of partial rows it wrote.
cudaError_t launch_adjoint_lorenz(int method, bool pp, int m, const AdjointArgs& a, int block, int num_sms,
                                  cudaStream_t s, int64_t* rows);
cudaError_t launch_adjoint_hh3(int method, bool pp, int m, const AdjointArgs& a, int block, int num_sms,
                               cudaStream_t s, int64_t* rows);
cudaError_t launch_adjoint_small(int rhs_id, int method, bool pp, int m, const AdjointArgs& a, int block,
                                 int num_sms, cudaStream_t s, int64_t* rows);
cudaError_t launch_adjoint_linear(int method, bool pp, int m, const AdjointArgs& a, int block, int num_sms,
                                  cudaStream_t s, int64_t* rows);
cudaError_t launch_batch_adjoint_linear(int method, bool pp, int m, const BatchAdjointArgs& b, int num_sms,
                                        cudaStream_t s);
cudaError_t launch_batch_adjoint_lorenz(int method, bool pp, int m, const BatchAdjointArgs& b, int num_sms,
                                        cudaStream_t s);
cudaError_t launch_batch_adjoint_hh3(int method, bool pp, int m, const BatchAdjointArgs& b, int num_sms,
                                     cudaStream_t s);
cudaError_t launch_batch_adjoint_small(int rhs_id, int method, bool pp, int m, const BatchAdjointArgs& b,
                                       int num_sms, cudaStream_t s);
// One batched-adjoint launch over b.tiles, then dp[m * np_stride + q] = sum of
// member m's rows in order, for m < n_members and q < n_params_kernel.
cudaError_t launch_batch_adjoint(int rhs_id, int method, bool pp, int m, const BatchAdjointArgs& b,
                                 const int* row0_dev, int n_members, int n_params_kernel, int num_sms,
                                 cudaStream_t s, double* dp_dev);

}  // namespace ff
