// ff_internal.h -- host-side internals shared by the C-ABI translation units:
// the system object, error reporting and small helpers.  Not part of the ABI.
#pragma once

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ff.h"
#include "ff_adjoint.h"
#include "ff_device.cuh"

namespace ff {

// Record the message returned by ff_last_error() on this thread and return `code`.
ff_status fail(ff_status code, const char* fmt, ...);
ff_status cuda_fail(cudaError_t e, const char* what);

struct Group {
    int64_t start, count;
    int64_t first, total;  // these particles are first .. first + count - 1 of a group of `total`
    int direction;
    uint64_t seed;
    double lo[FF_MAX_DIM], hi[FF_MAX_DIM];
};

// Makes a device current for the lifetime of the object and restores the caller's.
struct DeviceScope {
    int prev = -1;
    bool changed = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            changed = (err == cudaSuccess);
        }
    }
    ~DeviceScope() {
        if (changed) cudaSetDevice(prev);
    }
};

inline bool all_finite(const double* v, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace ff

struct ff_system {
    int device = 0;
    int num_sms = 1;
    cudaStream_t stream = nullptr;
    int rhs_id = 0, dim = 0, method = 0;
    unsigned flags = 0;
    int n_params = 0;
    double params[FF_MAX_PARAMS] = {};
    int64_t capacity = 0, pitch = 0, n_particles = 0;
    float* d_state = nullptr;
    float* d_comp = nullptr;
    float* d_pparam = nullptr;
    int pparam_index = -1;
    bool pparam_linspace = false;  // values monotone in the particle index
    int n_groups = 0;
    ff::Group groups[FF_MAX_GROUPS] = {};
    bool stepped = false;
    double t_fwd = 0, t_bwd = 0, c_fwd = 0, c_bwd = 0;  // Kahan-summed simulated time
    unsigned long long* d_counter = nullptr;
    uint32_t* d_stage = nullptr;  // device copy of a host image
    size_t stage_bytes = 0;
    // tiled sprite rendering: per-tile counts / offsets / cursors and the tile lists
    uint32_t* d_tiles = nullptr;
    size_t tiles_cap = 0;  // uint32 entries
    uint32_t* d_entries = nullptr;
    size_t entries_cap = 0;
    // launch shape
    int ppt = 1, block = 256, blocks_per_sm = 0;
    int64_t max_steps = 0;
    // particle reset
    int64_t steps_total = 0;  // steps since the last ff_reset (global step numbers)
    int check_every = 0;      // 0 = reset off
    double t_max = 0.0;
    bool has_bounds = false;
    float blo[FF_MAX_DIM] = {}, bhi[FF_MAX_DIM] = {};
    uint32_t* d_age = nullptr;
    uint32_t* d_resets = nullptr;
    ff::ResetTable* d_reset_table = nullptr;
    ff::ResetTable h_reset_table = {};
    bool reset_table_dirty = true;
    // adjoint tape
    bool tape_on = false;
    int64_t tape_every = 0, tape_slots = 0;
    int64_t ckpt_capacity = 0;  // checkpoint slots allocated (kept across tapes)
    float* d_ckpt = nullptr;
    ff::AdjChunk* d_chunks = nullptr;
    double* d_partial = nullptr;
    double* d_dp = nullptr;
    float* d_adj_scratch = nullptr;  // HH x 3 adjoint sweep: one chunk of stage points per thread
    size_t adj_scratch_floats = 0;
    int64_t partial_blocks = 0;
    std::vector<ff::AdjChunk> chunks;
    int64_t params_version = 0, chunk_version = -1;
    double chunk_dt = 0.0;
    // what the last ff_step / ff_step_splat launched (ff_last_launch)
    ff::LaunchRecord last_integrator{};
    int64_t last_integrator_launches = 0, last_splat_launches = 0;
    bool last_fused = false;
};

namespace ff {

// Kernel index of parameter q of the user's vector (LINEAR is padded to 8x8).
int kernel_param_index(const ff_system* s, int q);

// Argument block of an integrator launch with step dt for this system (no
// particle reset, no fused splat, n_steps left 0).
void fill_integrate_args(const ff_system* s, double dt, IntegrateArgs* a);

// Simulated-time and step bookkeeping after n_steps steps of size dt.
void account_steps(ff_system* s, int64_t n_steps, double dt);

}  // namespace ff
