// ff_api.cu -- the C ABI declared in include/ff.h: system ownership, argument
// checks, group tables, simulated time, and the launches of the hot-path
// kernels on the system's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cxxabi.h>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "ff.h"
#include "ff_adjoint.h"
#include "ff_aux.h"
#include "ff_device.cuh"
#include "ff_internal.h"

namespace {
thread_local std::string g_last_error;

int rhs_dim_ok(int rhs_id, int dim, int n_params) {
    switch (rhs_id) {
    case FF_RHS_LINEAR: return dim >= 1 && dim <= 8 && n_params == dim * dim;
    case FF_RHS_HARMONIC: return dim == 2 && n_params == 1;
    case FF_RHS_WILSON_COWAN: return dim == 2 && n_params == 10;
    case FF_RHS_LORENZ: return dim == 3 && n_params == 3;
    case FF_RHS_HH3: return dim == 15 && n_params == 16;
    default: return 0;
    }
}
}  // namespace

namespace ff {
ff_status fail(ff_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

ff_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(FF_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

int kernel_param_index(const ff_system* s, int q) {
    if (s->rhs_id == FF_RHS_LINEAR) return (q / s->dim) * 8 + (q % s->dim);
    return q;
}
}  // namespace ff

using ff::all_finite;
using ff::cuda_fail;
using ff::DeviceScope;
using ff::fail;
using ff::Group;
using ff::kernel_param_index;


namespace {

void kahan_add(double& sum, double& comp, double v) {
    double y = v - comp;
    double t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

ff_status seed_group(ff_system* s, const Group& g) {
    ff::SeedArgs a{};
    a.x = s->d_state;
    a.pitch = s->pitch;
    a.start = g.start;
    a.count = g.count;
    a.first = g.first;
    a.seed = g.seed;
    a.dim = s->dim;
    for (int k = 0; k < s->dim; ++k) {
        a.lo[k] = g.lo[k];
        a.width[k] = g.hi[k] - g.lo[k];
    }
    cudaError_t e = ff::launch_seed(a, s->num_sms, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "seed kernel launch");
    return FF_OK;
}

}  // namespace

extern "C" {

const char* ff_last_error(void) { return g_last_error.c_str(); }

ff_status ff_create_system(int rhs_id, int dim, const double* params, int n_params, int method,
                           unsigned flags, int64_t capacity, void* cuda_stream, ff_system** out) {
    if (!out) return fail(FF_ERR_INVALID_ARG, "ff_create_system: out is NULL");
    *out = nullptr;
    if (!rhs_dim_ok(rhs_id, dim, n_params))
        return fail(FF_ERR_INVALID_ARG, "ff_create_system: rhs_id %d does not take dim %d with %d params",
                    rhs_id, dim, n_params);
    if (method != FF_RK4 && method != FF_EULER)
        return fail(FF_ERR_INVALID_ARG, "ff_create_system: unknown method %d", method);
    if (flags & ~FF_FLAG_KAHAN) return fail(FF_ERR_INVALID_ARG, "ff_create_system: unknown flags 0x%x", flags);
    if (!params || !all_finite(params, n_params))
        return fail(FF_ERR_INVALID_ARG, "ff_create_system: params NULL or not finite");
    if (capacity < 1 || capacity > ((int64_t)1 << 40))
        return fail(FF_ERR_INVALID_ARG, "ff_create_system: capacity %lld out of range", (long long)capacity);
    ff_system* s = new (std::nothrow) ff_system();
    if (!s) return fail(FF_ERR_OOM, "ff_create_system: host allocation failed");
    cudaError_t e = cudaGetDevice(&s->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "ff_create_system: no usable CUDA device");
    }
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    s->rhs_id = rhs_id;
    s->dim = dim;
    s->method = method;
    s->flags = flags;
    s->n_params = n_params;
    memcpy(s->params, params, sizeof(double) * n_params);
    s->capacity = capacity;
    s->pitch = (capacity + 255) / 256 * 256;
    const size_t plane_bytes = sizeof(float) * (size_t)s->pitch;
    e = cudaMalloc(&s->d_state, plane_bytes * dim);
    if (e == cudaSuccess && (flags & FF_FLAG_KAHAN)) e = cudaMalloc(&s->d_comp, plane_bytes * dim);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_state, 0, plane_bytes * dim, s->stream);
    if (e == cudaSuccess && s->d_comp) e = cudaMemsetAsync(s->d_comp, 0, plane_bytes * dim, s->stream);
    if (e != cudaSuccess) {
        ff_status st = cuda_fail(e, "ff_create_system: device allocation");
        ff_destroy_system(s);
        return st;
    }
    // default launch shape: RK4 on Lorenz runs packed pairs, 4 particles per thread (2 when
    // compensated: its registers then leave room for more warps)
    const bool packed_lorenz = rhs_id == FF_RHS_LORENZ && method == FF_RK4;
    // HH3 plain RK4: two particles per thread, all three neurons of the pair packed
    const bool packed_hh3 = rhs_id == FF_RHS_HH3 && method == FF_RK4 && !(flags & FF_FLAG_KAHAN);
    s->ppt = packed_lorenz ? ((flags & FF_FLAG_KAHAN) ? 2 : 4) : (packed_hh3 ? 2 : 1);
    s->block = packed_lorenz ? 512 : 256;
    *out = s;
    return FF_OK;
}

ff_status ff_destroy_system(ff_system* s) {
    if (!s) return FF_OK;
    DeviceScope dev(s->device);
    cudaStreamSynchronize(s->stream);
    cudaFree(s->d_state);
    cudaFree(s->d_comp);
    cudaFree(s->d_pparam);
    cudaFree(s->d_counter);
    cudaFree(s->d_stage);
    cudaFree(s->d_tiles);
    cudaFree(s->d_entries);
    cudaFree(s->d_age);
    cudaFree(s->d_resets);
    cudaFree(s->d_reset_table);
    cudaFree(s->d_ckpt);
    cudaFree(s->d_chunks);
    cudaFree(s->d_partial);
    cudaFree(s->d_dp);
    cudaFree(s->d_adj_scratch);
    delete s;
    return FF_OK;
}

ff_status ff_seed_particles(ff_system* s, int64_t count, const double* lo, const double* hi,
                            int direction, uint64_t seed, int* group_id_out) {
    return ff_seed_particles_slice(s, count, 0, count, lo, hi, direction, seed, group_id_out);
}

ff_status ff_seed_particles_slice(ff_system* s, int64_t count, int64_t first, int64_t total, const double* lo,
                                  const double* hi, int direction, uint64_t seed, int* group_id_out) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_seed_particles: system is NULL");
    if (count >= 1 && (first < 0 || total < 1 || first > total - count))
        return fail(FF_ERR_INVALID_ARG, "ff_seed_particles_slice: slice [%lld, %lld) not inside a group of %lld",
                    (long long)first, (long long)(first + count), (long long)total);
    if (s->stepped) return fail(FF_ERR_STATE, "ff_seed_particles: system already stepped (call ff_reset first)");
    if (s->n_groups >= FF_MAX_GROUPS) return fail(FF_ERR_STATE, "ff_seed_particles: already %d groups", FF_MAX_GROUPS);
    if (count < 1) return fail(FF_ERR_INVALID_ARG, "ff_seed_particles: count %lld < 1", (long long)count);
    if (count > s->capacity - s->n_particles)
        return fail(FF_ERR_INVALID_ARG, "ff_seed_particles: %lld particles exceed the remaining capacity %lld",
                    (long long)count, (long long)(s->capacity - s->n_particles));
    if (!lo || !hi) return fail(FF_ERR_INVALID_ARG, "ff_seed_particles: lo/hi NULL");
    if (!all_finite(lo, s->dim) || !all_finite(hi, s->dim))
        return fail(FF_ERR_INVALID_ARG, "ff_seed_particles: non-finite box");
    for (int k = 0; k < s->dim; ++k)
        if (lo[k] > hi[k]) return fail(FF_ERR_INVALID_ARG, "ff_seed_particles: lo[%d] > hi[%d]", k, k);
    if (direction != 1 && direction != -1)
        return fail(FF_ERR_INVALID_ARG, "ff_seed_particles: direction %d is not +1 or -1", direction);
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_seed_particles: set device");
    Group g{};
    g.start = s->n_particles;
    g.count = count;
    g.first = first;
    g.total = total;
    g.direction = direction;
    g.seed = seed;
    for (int k = 0; k < s->dim; ++k) {
        g.lo[k] = lo[k];
        g.hi[k] = hi[k];
    }
    ff_status st = seed_group(s, g);
    if (st != FF_OK) return st;
    s->groups[s->n_groups] = g;
    if (group_id_out) *group_id_out = s->n_groups;
    s->n_groups++;
    s->n_particles += count;
    s->reset_table_dirty = true;
    return FF_OK;
}

static ff_status clear_reset_state(ff_system* s) {
    if (!s->d_age) return FF_OK;
    cudaError_t e = cudaMemsetAsync(s->d_age, 0, sizeof(uint32_t) * (size_t)s->pitch, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_resets, 0, sizeof(uint32_t) * (size_t)s->pitch, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing particle ages");
    return FF_OK;
}

ff_status ff_reset(ff_system* s) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_reset: system is NULL");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_reset: set device");
    for (int g = 0; g < s->n_groups; ++g) {
        ff_status st = seed_group(s, s->groups[g]);
        if (st != FF_OK) return st;
    }
    if (s->d_comp) {
        cudaError_t e = cudaMemsetAsync(s->d_comp, 0, sizeof(float) * (size_t)s->pitch * s->dim, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "ff_reset: clear compensation");
    }
    s->t_fwd = s->t_bwd = s->c_fwd = s->c_bwd = 0.0;
    s->stepped = false;
    s->steps_total = 0;
    s->tape_on = false;  // the state the tape started from is gone
    ff_status st = clear_reset_state(s);
    if (st != FF_OK) return st;
    return FF_OK;
}

static ff_status ensure_pparam(ff_system* s) {
    if (s->d_pparam) return FF_OK;
    cudaError_t e = cudaMalloc(&s->d_pparam, sizeof(float) * (size_t)s->pitch);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->d_pparam, 0, sizeof(float) * (size_t)s->pitch, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "per-particle parameter allocation");
    return FF_OK;
}

ff_status ff_set_particle_param(ff_system* s, int param_index, double lo, double hi) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param: system is NULL");
    return ff_set_particle_param_slice(s, param_index, lo, hi, 0, s->n_particles);
}

ff_status ff_set_particle_param_slice(ff_system* s, int param_index, double lo, double hi, int64_t first,
                                      int64_t total) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param: system is NULL");
    if (param_index == -1) {
        s->pparam_index = -1;
        s->params_version++;
        return FF_OK;
    }
    if (param_index < 0 || param_index >= s->n_params)
        return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param: index %d out of range", param_index);
    if (!std::isfinite(lo) || !std::isfinite(hi))
        return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param: non-finite bounds");
    if (s->n_particles < 1) return fail(FF_ERR_STATE, "ff_set_particle_param: no particles seeded");
    if (first < 0 || first > total - s->n_particles)
        return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param_slice: particles [%lld, %lld) not inside %lld",
                    (long long)first, (long long)(first + s->n_particles), (long long)total);
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_set_particle_param: set device");
    ff_status st = ensure_pparam(s);
    if (st != FF_OK) return st;
    cudaError_t e = ff::launch_linspace(s->d_pparam, s->n_particles, lo, hi, first, total, s->num_sms, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "linspace kernel launch");
    s->pparam_index = param_index;
    s->pparam_linspace = true;
    s->params_version++;
    return FF_OK;
}

ff_status ff_set_particle_param_values(ff_system* s, int param_index, const float* values,
                                       int values_is_device) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param_values: system is NULL");
    if (param_index < 0 || param_index >= s->n_params)
        return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param_values: index %d out of range", param_index);
    if (!values) return fail(FF_ERR_INVALID_ARG, "ff_set_particle_param_values: values is NULL");
    if (s->n_particles < 1) return fail(FF_ERR_STATE, "ff_set_particle_param_values: no particles seeded");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_set_particle_param_values: set device");
    ff_status st = ensure_pparam(s);
    if (st != FF_OK) return st;
    cudaError_t e = cudaMemcpyAsync(s->d_pparam, values, sizeof(float) * (size_t)s->n_particles,
                                    values_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    s->stream);
    if (e == cudaSuccess && !values_is_device) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_set_particle_param_values: copy");
    s->pparam_index = param_index;
    s->pparam_linspace = false;
    s->params_version++;
    return FF_OK;
}

ff_status ff_get_particle_param(ff_system* s, float* dst, int dst_is_device, int* param_index_out) {
    if (!s || !dst) return fail(FF_ERR_INVALID_ARG, "ff_get_particle_param: NULL argument");
    if (!s->d_pparam) return fail(FF_ERR_STATE, "ff_get_particle_param: no per-particle parameter set");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_get_particle_param: set device");
    cudaError_t e = cudaMemcpyAsync(dst, s->d_pparam, sizeof(float) * (size_t)s->n_particles,
                                    dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess && !dst_is_device) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_get_particle_param: copy");
    if (param_index_out) *param_index_out = s->pparam_index;
    return FF_OK;
}

ff_status ff_set_params(ff_system* s, const double* params, int n_params) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_set_params: system is NULL");
    if (!params || n_params != s->n_params)
        return fail(FF_ERR_INVALID_ARG, "ff_set_params: expected %d params", s->n_params);
    if (!all_finite(params, n_params)) return fail(FF_ERR_INVALID_ARG, "ff_set_params: non-finite values");
    // Parameters travel by value in each launch's argument block, so the new
    // values are seen exactly by the launches enqueued after this call.
    memcpy(s->params, params, sizeof(double) * n_params);
    s->params_version++;
    return FF_OK;
}

ff_status ff_set_launch(ff_system* s, int ppt, int block, int blocks_per_sm, int64_t max_steps) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_set_launch: system is NULL");
    if (ppt == 0) ppt = s->ppt;
    if (block == 0) block = s->block;
    if (ppt != 1 && ppt != 2 && ppt != 4) return fail(FF_ERR_INVALID_ARG, "ff_set_launch: ppt %d not 1, 2 or 4", ppt);
    if (ppt != 1 && s->dim > 4 && s->rhs_id != FF_RHS_LINEAR && !(s->rhs_id == FF_RHS_HH3 && ppt == 2))
        return fail(FF_ERR_INVALID_ARG, "ff_set_launch: ppt > 1 needs dim <= 4 (HH3: ppt 2)");
    if (ppt != 1 && s->rhs_id == FF_RHS_LINEAR) return fail(FF_ERR_INVALID_ARG, "ff_set_launch: LINEAR runs ppt 1");
    if (block < 32 || block > 1024 || block % 32) return fail(FF_ERR_INVALID_ARG, "ff_set_launch: block %d", block);
    if (blocks_per_sm < 0 || blocks_per_sm > 64) return fail(FF_ERR_INVALID_ARG, "ff_set_launch: blocks_per_sm %d", blocks_per_sm);
    if (max_steps < 0) return fail(FF_ERR_INVALID_ARG, "ff_set_launch: max_steps < 0");
    s->ppt = ppt;
    s->block = block;
    s->blocks_per_sm = blocks_per_sm;
    s->max_steps = max_steps;
    return FF_OK;
}

ff_status ff_set_reset(ff_system* s, const double* bound_lo, const double* bound_hi, double t_max,
                       int check_every) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_set_reset: system is NULL");
    if (check_every < 0) return fail(FF_ERR_INVALID_ARG, "ff_set_reset: check_every < 0");
    if ((bound_lo == nullptr) != (bound_hi == nullptr))
        return fail(FF_ERR_INVALID_ARG, "ff_set_reset: give both bounds or neither");
    if (!std::isfinite(t_max)) return fail(FF_ERR_INVALID_ARG, "ff_set_reset: t_max not finite");
    if (bound_lo) {
        if (!all_finite(bound_lo, s->dim) || !all_finite(bound_hi, s->dim))
            return fail(FF_ERR_INVALID_ARG, "ff_set_reset: non-finite bounds");
        for (int k = 0; k < s->dim; ++k)
            if (bound_lo[k] > bound_hi[k]) return fail(FF_ERR_INVALID_ARG, "ff_set_reset: bound_lo[%d] > bound_hi[%d]", k, k);
    }
    if (check_every > 0 && s->tape_on)
        return fail(FF_ERR_UNSUPPORTED, "ff_set_reset: particle reset cannot be taped for the adjoint");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_set_reset: set device");
    if (check_every > 0 && !s->d_age) {
        const size_t n = sizeof(uint32_t) * (size_t)s->pitch;
        cudaError_t e = cudaMalloc(&s->d_age, n);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_resets, n);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_reset_table, sizeof(ff::ResetTable));
        if (e == cudaSuccess) e = cudaMemsetAsync(s->d_age, 0, n, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->d_resets, 0, n, s->stream);
        if (e != cudaSuccess) {
            cudaFree(s->d_age);
            cudaFree(s->d_resets);
            cudaFree(s->d_reset_table);
            s->d_age = s->d_resets = nullptr;
            s->d_reset_table = nullptr;
            return cuda_fail(e, "ff_set_reset: allocation");
        }
    }
    s->check_every = check_every;
    s->t_max = t_max;
    s->has_bounds = bound_lo != nullptr;
    for (int k = 0; k < s->dim; ++k) {
        s->blo[k] = bound_lo ? (float)bound_lo[k] : 0.0f;
        s->bhi[k] = bound_hi ? (float)bound_hi[k] : 0.0f;
    }
    s->reset_table_dirty = true;
    return FF_OK;
}

ff_status ff_get_reset_state(ff_system* s, uint32_t* age, uint32_t* resets, int dst_is_device) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_get_reset_state: system is NULL");
    if (!s->d_age) return fail(FF_ERR_STATE, "ff_get_reset_state: the reset was never enabled");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_get_reset_state: set device");
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t n = sizeof(uint32_t) * (size_t)s->n_particles;
    cudaError_t e = cudaSuccess;
    if (age && n) e = cudaMemcpyAsync(age, s->d_age, n, kind, s->stream);
    if (e == cudaSuccess && resets && n) e = cudaMemcpyAsync(resets, s->d_resets, n, kind, s->stream);
    if (e == cudaSuccess && !dst_is_device) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_get_reset_state: copy");
    return FF_OK;
}

static ff_status upload_reset_table(ff_system* s) {
    ff::ResetTable& t = s->h_reset_table;
    t = ff::ResetTable{};
    for (int g = 0; g < s->n_groups; ++g) {
        for (int k = 0; k < s->dim; ++k) {
            t.lo[g][k] = s->groups[g].lo[k];
            t.width[g][k] = s->groups[g].hi[k] - s->groups[g].lo[k];
        }
        t.count[g] = s->groups[g].total;
        t.first[g] = s->groups[g].first;
        t.seed[g] = s->groups[g].seed;
    }
    for (int k = 0; k < s->dim; ++k) {
        t.blo[k] = s->blo[k];
        t.bhi[k] = s->bhi[k];
    }
    t.has_bounds = s->has_bounds ? 1 : 0;
    // pageable source: the call returns once the table has been staged, so later edits are safe
    cudaError_t e = cudaMemcpyAsync(s->d_reset_table, &t, sizeof(t), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_step: reset table upload");
    s->reset_table_dirty = false;
    return FF_OK;
}

// Launch the integrator for n_steps steps of size dt (no argument checks).  With
// `fuse`, the last launch also projects and splats the final states (the caller
// checked that the group-uniform packed kernel runs).
}  // extern "C"

namespace ff {
void fill_integrate_args(const ff_system* s, double dt, IntegrateArgs* out) {
    IntegrateArgs a{};
    a.x = s->d_state;
    a.comp = s->d_comp;
    a.pparam = s->d_pparam;
    a.pitch = s->pitch;
    a.dim = s->dim;
    a.n_groups = s->n_groups;
    a.pidx = s->pparam_index >= 0 ? kernel_param_index(s, s->pparam_index) : -1;
    // all processed particles are a multiple of 4 (<= pitch): every vector access stays in bounds
    const int64_t n_work = (s->n_particles + 3) / 4 * 4;
    for (int g = 0; g < s->n_groups; ++g) {
        a.gstart[g] = s->groups[g].start;
        a.gend[g] = (g + 1 < s->n_groups) ? s->groups[g + 1].start : n_work;
        a.gh[g] = (float)(s->groups[g].direction * dt);
    }
    for (int q = 0; q < s->n_params; ++q) a.p[kernel_param_index(s, q)] = (float)s->params[q];
    a.n_vec = n_work / s->ppt;
    a.n_real = s->n_particles;
    *out = a;
}

void account_steps(ff_system* s, int64_t n_steps, double dt) {
    bool any_fwd = false, any_bwd = false;
    for (int g = 0; g < s->n_groups; ++g) (s->groups[g].direction > 0 ? any_fwd : any_bwd) = true;
    const double span = (double)n_steps * dt;
    if (any_fwd) kahan_add(s->t_fwd, s->c_fwd, span);
    if (any_bwd) kahan_add(s->t_bwd, s->c_bwd, -span);
    s->stepped = true;
}
}  // namespace ff

extern "C" {

// Checkpoints of a taped call: before step first + k * every of the call (k < count)
// the state goes to checkpoint slot slot0 + k.
struct TapePlan {
    int64_t first, every, count;
    int slot0;
};

static ff_status integrate_steps(ff_system* s, int64_t n_steps, double dt, const ff::ViewArgs* fuse = nullptr,
                                 const TapePlan* tape = nullptr) {
    ff::IntegrateArgs a{};
    ff::fill_integrate_args(s, dt, &a);
    const int ppt = s->ppt;
    ff::LaunchShape shape{ppt, s->block, s->blocks_per_sm, s->num_sms};
    const bool kahan = (s->flags & FF_FLAG_KAHAN) != 0;
    const bool pp = s->pparam_index >= 0;
    if (s->check_every > 0) {
        if (s->reset_table_dirty) {
            ff_status st = upload_reset_table(s);
            if (st != FF_OK) return st;
        }
        a.reset = s->d_reset_table;
        a.age = s->d_age;
        a.resets = s->d_resets;
        a.check_every = s->check_every;
        const double steps = (s->t_max > 0.0 && dt != 0.0) ? std::ceil(s->t_max / std::fabs(dt)) : 0.0;
        a.max_age = steps <= 0.0 ? 0u : (steps >= 4294967295.0 ? 4294967295u : (uint32_t)steps);
    }
    int64_t left = n_steps;
    s->last_integrator_launches = 0;
    s->last_splat_launches = 0;
    s->last_fused = false;
    while (left > 0) {
        int64_t chunk = (s->max_steps > 0 && left > s->max_steps) ? s->max_steps : left;
        if (chunk > ((int64_t)1 << 30)) chunk = (int64_t)1 << 30;  // kernels count steps in 32 bits
        a.n_steps = chunk;
        a.step0 = s->steps_total;
        a.ckpt = nullptr;
        if (tape && tape->count > 0) {
            // the plan's first checkpoint at or after this launch's first step
            const int64_t done = n_steps - left;
            const int64_t k0 = done <= tape->first ? 0 : (done - tape->first + tape->every - 1) / tape->every;
            const int64_t at = tape->first + k0 * tape->every;
            if (k0 < tape->count && at < done + chunk) {
                a.ckpt = s->d_ckpt;
                a.ck_stride = (int64_t)s->dim * s->pitch;
                a.ck_first = (int)(at - done);
                a.ck_every = (int)tape->every;
                a.ck_slot0 = tape->slot0 + (int)k0;
            }
        }
        cudaError_t e;
        ff::last_launch_record() = ff::LaunchRecord{};
        const bool fused = fuse && chunk == left;
        if (fused) {
            a.view = *fuse;
            e = ff::launch_integrate_lorenz_splat(pp, a, shape, s->stream);
        } else {
            e = ff::launch_integrate(s->rhs_id, s->method, kahan, pp, a, shape, s->stream);
        }
        if (e != cudaSuccess) return cuda_fail(e, "integrator launch");
        if (ff::last_launch_record().kernel) {
            s->last_integrator = ff::last_launch_record();
            s->last_integrator_launches += 1;
            s->last_fused = fused;
        }
        left -= chunk;
        s->steps_total += chunk;
    }
    return FF_OK;
}

// Taped stepping: a checkpoint of the state at the start of every chunk; a chunk
// ends after tape_every steps or when the parameters or dt change.  The integrator
// writes the checkpoints inside its launches (run_steps), so a call is as many
// launches as an untaped one.  The tape's capacity is checked before any step.
static ff_status taped_steps(ff_system* s, int64_t n_steps, double dt) {
    const bool open = !s->chunks.empty() && s->chunk_version == s->params_version && s->chunk_dt == dt;
    int64_t cont = open ? s->tape_every - s->chunks.back().n_steps : 0;  // steps left in the open chunk
    if (cont > n_steps) cont = n_steps;
    const int64_t rest = n_steps - cont;
    const int64_t fresh = (rest + s->tape_every - 1) / s->tape_every;  // chunks this call starts
    if ((int64_t)s->chunks.size() + fresh > s->tape_slots)
        return fail(FF_ERR_STATE, "ff_step: the tape is full (raise max_steps in ff_tape_begin)");
    const TapePlan plan{cont, s->tape_every, fresh, (int)s->chunks.size()};
    ff_status st = integrate_steps(s, n_steps, dt, nullptr, &plan);
    if (st != FF_OK) return st;
    if (cont > 0) s->chunks.back().n_steps += (int)cont;
    for (int64_t k = 0; k < fresh; ++k) {
        ff::AdjChunk c{};
        c.ckpt = plan.slot0 + (int)k;
        const int64_t left = rest - k * s->tape_every;
        c.n_steps = (int)(left < s->tape_every ? left : s->tape_every);
        for (int q = 0; q < s->n_params; ++q) c.p[kernel_param_index(s, q)] = (float)s->params[q];
        for (int g = 0; g < s->n_groups; ++g) c.gh[g] = (float)(s->groups[g].direction * dt);
        s->chunks.push_back(c);
    }
    s->chunk_version = s->params_version;
    s->chunk_dt = dt;
    return FF_OK;
}

ff_status ff_step(ff_system* s, int64_t n_steps, double dt) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_step: system is NULL");
    if (n_steps < 0) return fail(FF_ERR_INVALID_ARG, "ff_step: n_steps %lld < 0", (long long)n_steps);
    if (!std::isfinite(dt)) return fail(FF_ERR_INVALID_ARG, "ff_step: dt not finite");
    if (s->n_particles < 1) return fail(FF_ERR_STATE, "ff_step: no particles seeded");
    if (n_steps == 0) return FF_OK;
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_step: set device");
    ff_status st = s->tape_on ? taped_steps(s, n_steps, dt) : integrate_steps(s, n_steps, dt);
    if (st != FF_OK) return st;
    ff::account_steps(s, n_steps, dt);
    return FF_OK;
}

static void free_tape(ff_system* s) {
    cudaFree(s->d_ckpt);
    cudaFree(s->d_chunks);
    cudaFree(s->d_partial);
    cudaFree(s->d_dp);
    cudaFree(s->d_adj_scratch);
    s->d_ckpt = nullptr;
    s->d_chunks = nullptr;
    s->d_partial = nullptr;
    s->d_dp = nullptr;
    s->d_adj_scratch = nullptr;
    s->adj_scratch_floats = 0;
    s->ckpt_capacity = 0;
    s->chunks.clear();
    s->tape_on = false;
}

ff_status ff_tape_begin(ff_system* s, int64_t checkpoint_every, int64_t max_steps) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_tape_begin: system is NULL");
    if (checkpoint_every < 1 || checkpoint_every > 256)
        return fail(FF_ERR_INVALID_ARG, "ff_tape_begin: checkpoint_every must be 1..256");
    if (max_steps < 1) return fail(FF_ERR_INVALID_ARG, "ff_tape_begin: max_steps < 1");
    if (!ff::adjoint_supported(s->rhs_id))
        return fail(FF_ERR_UNSUPPORTED, "ff_tape_begin: no adjoint for this system yet");
    if (s->check_every > 0) return fail(FF_ERR_UNSUPPORTED, "ff_tape_begin: particle reset is on");
    if (s->n_particles < 1) return fail(FF_ERR_STATE, "ff_tape_begin: no particles seeded");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_tape_begin: set device");
    const int64_t slots = (max_steps + checkpoint_every - 1) / checkpoint_every + 16;
    if (s->d_ckpt && s->ckpt_capacity >= slots) {
        // the previous tape's buffers are large enough: reuse them (work that still reads
        // them is ordered before the new tape's steps on the system's stream)
        s->chunks.clear();
    } else {
        cudaError_t e = cudaStreamSynchronize(s->stream);  // earlier work may still read the old tape
        if (e != cudaSuccess) return cuda_fail(e, "ff_tape_begin: synchronise");
        free_tape(s);
        s->partial_blocks = ff::adjoint_partial_rows(s->num_sms);
        e = cudaMalloc(&s->d_ckpt, sizeof(float) * (size_t)slots * s->dim * s->pitch);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_chunks, sizeof(ff::AdjChunk) * (size_t)slots);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_partial, sizeof(double) * (size_t)s->partial_blocks * FF_MAX_PARAMS);
        if (e == cudaSuccess) e = cudaMalloc(&s->d_dp, sizeof(double) * FF_MAX_PARAMS);
        if (e != cudaSuccess) {
            free_tape(s);
            return cuda_fail(e, "ff_tape_begin: allocation");
        }
        s->ckpt_capacity = slots;
    }
    s->tape_every = checkpoint_every;
    s->tape_slots = slots;
    s->chunk_version = -1;
    s->tape_on = true;
    return FF_OK;
}

ff_status ff_tape_end(ff_system* s) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_tape_end: system is NULL");
    DeviceScope dev(s->device);
    cudaStreamSynchronize(s->stream);
    free_tape(s);
    return FF_OK;
}

ff_status ff_backward(ff_system* s, const float* dL_dxT_dev, float* dL_dx0_dev, double* dL_dp_host) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_backward: system is NULL");
    if (!dL_dxT_dev || !dL_dx0_dev || !dL_dp_host) return fail(FF_ERR_INVALID_ARG, "ff_backward: NULL buffer");
    if (!s->tape_on) return fail(FF_ERR_STATE, "ff_backward: no tape (call ff_tape_begin before stepping)");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_backward: set device");
    double dp[FF_MAX_PARAMS] = {};
    if (s->chunks.empty()) {  // nothing taped: the map is the identity
        cudaError_t e = cudaMemcpyAsync(dL_dx0_dev, dL_dxT_dev, sizeof(float) * (size_t)s->dim * s->n_particles,
                                        cudaMemcpyDeviceToDevice, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "ff_backward: copy");
        for (int q = 0; q < s->n_params; ++q) dL_dp_host[q] = 0.0;
        return FF_OK;
    }
    cudaError_t e = cudaMemcpyAsync(s->d_chunks, s->chunks.data(), sizeof(ff::AdjChunk) * s->chunks.size(),
                                    cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_backward: chunk table upload");
    ff::AdjointArgs a{};
    a.ckpt = s->d_ckpt;
    a.chunks = s->d_chunks;
    a.n_chunks = (int)s->chunks.size();
    a.dim = s->dim;
    a.lam_in = dL_dxT_dev;
    a.lam_out = dL_dx0_dev;
    a.pparam = s->d_pparam;
    a.pidx = s->pparam_index >= 0 ? kernel_param_index(s, s->pparam_index) : -1;
    a.np_stride = FF_MAX_PARAMS;
    a.partial = s->d_partial;
    a.max_blocks = s->partial_blocks / 8;  // room for 8 rows (warps) per block
    a.n = s->n_particles;
    a.pitch = s->pitch;
    a.n_groups = s->n_groups;
    a.max_chunk = (int)s->tape_every;
    for (int g = 0; g < s->n_groups; ++g) a.gstart[g] = s->groups[g].start;
    // the HH x 3 sweep keeps a chunk of stage points per thread in a scratch area,
    // allocated on first use and kept with the tape
    const int64_t scratch_threads =
        ff::adjoint_scratch_threads(s->rhs_id, s->method, s->pparam_index >= 0, s->num_sms, false);
    if (scratch_threads > 0) {
        const size_t need = (size_t)scratch_threads * (size_t)s->tape_every *
                            (size_t)ff::adjoint_scratch_floats_per_step(s->rhs_id, s->method);
        if (need > s->adj_scratch_floats) {
            cudaFree(s->d_adj_scratch);  // waits for any sweep still reading it
            s->d_adj_scratch = nullptr;
            s->adj_scratch_floats = 0;
            e = cudaMalloc(&s->d_adj_scratch, sizeof(float) * need);
            if (e != cudaSuccess) return cuda_fail(e, "ff_backward: scratch allocation");
            s->adj_scratch_floats = need;
        }
        a.scratch = s->d_adj_scratch;
        a.scratch_threads = scratch_threads;
    }
    const int np_kernel = s->rhs_id == FF_RHS_LINEAR ? 64 : s->n_params;
    e = ff::launch_adjoint(s->rhs_id, s->method, s->pparam_index >= 0, ff::adjoint_sub_steps(s->tape_every), a,
                           s->num_sms, s->stream, s->d_dp, np_kernel);
    if (e != cudaSuccess) return cuda_fail(e, "ff_backward: adjoint launch");
    e = cudaMemcpyAsync(dp, s->d_dp, sizeof(double) * np_kernel, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_backward: gradient download");
    for (int q = 0; q < s->n_params; ++q) dL_dp_host[q] = dp[kernel_param_index(s, q)];
    return FF_OK;
}

// The device image a render call draws into: the caller's device image, or the
// system's staging buffer holding (when accumulating) a copy of the caller's host
// image; cleared first unless accumulating.
static ff_status image_begin(ff_system* s, void* image, int image_is_device, size_t bytes, int accumulate,
                             void** target, const char* who) {
    cudaError_t e = cudaSuccess;
    *target = image;
    if (!image_is_device) {
        if (s->stage_bytes < bytes) {
            cudaFree(s->d_stage);
            s->d_stage = nullptr;
            s->stage_bytes = 0;
            e = cudaMalloc(&s->d_stage, bytes);
            if (e != cudaSuccess) return cuda_fail(e, who);
            s->stage_bytes = bytes;
        }
        *target = s->d_stage;
        if (accumulate) e = cudaMemcpyAsync(*target, image, bytes, cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess && !accumulate) e = cudaMemsetAsync(*target, 0, bytes, s->stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return FF_OK;
}

// After the render kernels: a host image is copied back (and the call synchronises).
static ff_status image_end(ff_system* s, void* image, int image_is_device, size_t bytes, void* target,
                           const char* who) {
    if (image_is_device) return FF_OK;
    cudaError_t e = cudaMemcpyAsync(image, target, bytes, cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, who);
    return FF_OK;
}

// Checked view -> kernel view arguments (axes, window or camera, image size, group mask).
static ff_status view_args(const ff_system* s, const ff_view* v, ff::ViewArgs* out) {
    ff::ViewArgs a{};
    if (v->ndim_view != 2 && v->ndim_view != 3)
        return fail(FF_ERR_INVALID_ARG, "ff_project_splat: ndim_view %d not 2 or 3", v->ndim_view);
    if (v->width < 1 || v->height < 1 || (int64_t)v->width * v->height >= ((int64_t)1 << 31))
        return fail(FF_ERR_INVALID_ARG, "ff_project_splat: image %d x %d out of range", v->width, v->height);
    for (int q = 0; q < v->ndim_view; ++q) {
        const int ax = v->axes[q];
        if (ax < 0 || ax > s->dim || (ax == s->dim && s->pparam_index < 0))
            return fail(FF_ERR_INVALID_ARG, "ff_project_splat: axis %d out of range", ax);
        a.axes[q] = ax;
    }
    a.ndim = v->ndim_view;
    a.W = v->width;
    a.H = v->height;
    a.Wf = (float)v->width;
    a.Hf = (float)v->height;
    if (v->ndim_view == 2) {
        for (int q = 0; q < 2; ++q)
            if (!std::isfinite(v->lo[q]) || !std::isfinite(v->hi[q]) || !(v->lo[q] < v->hi[q]))
                return fail(FF_ERR_INVALID_ARG, "ff_project_splat: window axis %d needs finite lo < hi", q);
        a.lo0 = (float)v->lo[0];
        a.lo1 = (float)v->lo[1];
        a.s0 = (float)((double)v->width / (v->hi[0] - v->lo[0]));
        a.s1 = (float)((double)v->height / (v->hi[1] - v->lo[1]));
    } else {
        for (int q = 0; q < 16; ++q) {
            if (!std::isfinite(v->mvp[q])) return fail(FF_ERR_INVALID_ARG, "ff_project_splat: non-finite mvp");
            a.m[q] = v->mvp[q];
        }
        a.lo0 = a.lo1 = -1.0f;
        a.s0 = (float)((double)v->width / 2.0);
        a.s1 = (float)((double)v->height / 2.0);
    }
    const uint32_t all = (s->n_groups >= 32) ? 0xffffffffu : ((1u << s->n_groups) - 1u);
    a.mask = v->group_mask & all;
    *out = a;
    return FF_OK;
}

ff_status ff_project_splat(ff_system* s, const ff_view* v, uint32_t* image, int image_is_device) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_project_splat: system is NULL");
    if (!v || !image) return fail(FF_ERR_INVALID_ARG, "ff_project_splat: view or image is NULL");
    ff::SplatArgs a{};
    ff_status vst = view_args(s, v, &a.v);
    if (vst != FF_OK) return vst;
    for (int q = 0; q < v->ndim_view; ++q)
        a.ax[q] = (a.v.axes[q] == s->dim) ? s->d_pparam : s->d_state + (int64_t)a.v.axes[q] * s->pitch;
    a.n = s->n_particles;
    a.n_groups = s->n_groups;
    uint32_t all = (s->n_groups >= 32) ? 0xffffffffu : ((1u << s->n_groups) - 1u);
    for (int g = 0; g < s->n_groups; ++g) a.gstart[g] = s->groups[g].start;
    const bool masked = a.v.mask != all;

    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_project_splat: set device");
    const size_t bytes = sizeof(uint32_t) * (size_t)v->width * v->height;
    void* target = nullptr;
    ff_status st = image_begin(s, image, image_is_device, bytes, v->accumulate, &target, "ff_project_splat");
    if (st != FF_OK) return st;
    cudaError_t e = cudaSuccess;
    a.v.image = static_cast<uint32_t*>(target);
    bool strip = false;  // a linspace parameter on an axis: consecutive particles share a column or row
    for (int q = 0; q < v->ndim_view; ++q) strip = strip || (v->axes[q] == s->dim && s->pparam_linspace);
    s->last_splat_launches = 0;
    if (s->n_particles > 0 && a.v.mask != 0) {
        e = ff::launch_splat(a, v->ndim_view, masked, strip, s->num_sms, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "splat kernel launch");
        s->last_splat_launches = 1;
    }
    return image_end(s, image, image_is_device, bytes, target, "ff_project_splat");
}

ff_status ff_project_sprites(ff_system* s, const ff_view* v, const ff_sprite* sp, float* image,
                             int image_is_device) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_project_sprites: system is NULL");
    if (!v || !image || !sp) return fail(FF_ERR_INVALID_ARG, "ff_project_sprites: view, sprite or image is NULL");
    if (!(sp->radius > 0.0f && sp->radius <= FF_SPRITE_MAX_RADIUS))
        return fail(FF_ERR_INVALID_ARG, "ff_project_sprites: radius %g outside (0, 32]", (double)sp->radius);
    if (!std::isfinite(sp->gain)) return fail(FF_ERR_INVALID_ARG, "ff_project_sprites: non-finite gain");
    if (sp->technique < FF_SPRITE_AUTO || sp->technique > FF_SPRITE_TILED)
        return fail(FF_ERR_INVALID_ARG, "ff_project_sprites: technique %d unknown", sp->technique);
    if (image_is_device && (reinterpret_cast<uintptr_t>(image) & 15u) != 0)
        return fail(FF_ERR_INVALID_ARG, "ff_project_sprites: device image not aligned to 16 bytes");
    ff::SpriteArgs a{};
    ff_status vst = view_args(s, v, &a.v);
    if (vst != FF_OK) return vst;
    for (int g = 0; g < FF_MAX_GROUPS; ++g) {
        float c[4];
        for (int k = 0; k < 4; ++k) {
            if (!std::isfinite(sp->colour[g][k]))
                return fail(FF_ERR_INVALID_ARG, "ff_project_sprites: non-finite colour of group %d", g);
            c[k] = sp->gain * sp->colour[g][k];
        }
        a.colour[g] = make_float4(c[0], c[1], c[2], c[3]);
    }
    for (int q = 0; q < v->ndim_view; ++q)
        a.ax[q] = (a.v.axes[q] == s->dim) ? s->d_pparam : s->d_state + (int64_t)a.v.axes[q] * s->pitch;
    a.n = s->n_particles;
    a.n_groups = s->n_groups;
    for (int g = 0; g < s->n_groups; ++g) a.gstart[g] = s->groups[g].start;
    a.R = sp->radius;
    a.inv_r2 = (float)(1.0 / ((double)sp->radius * (double)sp->radius));
    const uint32_t all = (s->n_groups >= 32) ? 0xffffffffu : ((1u << s->n_groups) - 1u);
    const bool masked = a.v.mask != all;
    // tiled where it applies: the per-tile histograms fit, the tile lists index in 32 bits
    // (decided before any device work, so a rejected call leaves the image untouched)
    const int n_tiles = ff::sprite_tiles(v->width, v->height);
    const int64_t entries = ff::sprite_entries_bound(s->n_particles, sp->radius);
    const bool tiles_fit = n_tiles <= ff::kSpriteMaxTiles && entries < ((int64_t)1 << 31);
    if (sp->technique == FF_SPRITE_TILED && !tiles_fit)
        return fail(FF_ERR_UNSUPPORTED, "ff_project_sprites: %d tiles, more than the tiled technique takes", n_tiles);
    // AUTO takes the direct technique: measured faster on every workload tried (the L2's
    // vector reductions outrun shared-memory atomics on the dense tiles of an attractor)
    const bool tiled = sp->technique == FF_SPRITE_TILED;

    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_project_sprites: set device");
    const size_t bytes = sizeof(float) * 4 * (size_t)v->width * v->height;
    void* target = nullptr;
    ff_status ist = image_begin(s, image, image_is_device, bytes, v->accumulate, &target, "ff_project_sprites");
    if (ist != FF_OK) return ist;
    cudaError_t e = cudaSuccess;
    a.image = static_cast<float4*>(target);
    if (tiled) {
        const size_t need_tiles = 4 * (size_t)n_tiles + 2;
        if (s->tiles_cap < need_tiles) {
            cudaFree(s->d_tiles);
            s->d_tiles = nullptr;
            s->tiles_cap = 0;
            e = cudaMalloc(&s->d_tiles, sizeof(uint32_t) * need_tiles);
            if (e != cudaSuccess) return cuda_fail(e, "ff_project_sprites: tile table");
            s->tiles_cap = need_tiles;
        }
        if (s->entries_cap < (size_t)entries) {
            cudaFree(s->d_entries);
            s->d_entries = nullptr;
            s->entries_cap = 0;
            e = cudaMalloc(&s->d_entries, sizeof(uint32_t) * (size_t)entries);
            if (e != cudaSuccess) return cuda_fail(e, "ff_project_sprites: tile lists");
            s->entries_cap = (size_t)entries;
        }
    }
    if (s->n_particles > 0 && a.v.mask != 0) {
        e = tiled ? ff::launch_sprites_tiled(a, v->ndim_view, masked, s->d_tiles, s->d_entries, s->num_sms, s->stream)
                  : ff::launch_sprites(a, v->ndim_view, masked, s->num_sms, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sprite kernel launch");
    }
    return image_end(s, image, image_is_device, bytes, target, "ff_project_sprites");
}

ff_status ff_step_splat(ff_system* s, int64_t n_steps, double dt, const ff_view* v, uint32_t* image,
                        int image_is_device) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_step_splat: system is NULL");
    if (!v || !image) return fail(FF_ERR_INVALID_ARG, "ff_step_splat: view or image is NULL");
    ff::ViewArgs va{};
    ff_status st = view_args(s, v, &va);
    if (st != FF_OK) return st;
    // the fused path: group-uniform packed Lorenz kernel, device image, plain stepping
    ff::IntegrateArgs probe{};
    probe.n_groups = s->n_groups;
    for (int g = 0; g < s->n_groups; ++g) probe.gstart[g] = s->groups[g].start;
    probe.pidx = s->pparam_index >= 0 ? kernel_param_index(s, s->pparam_index) : -1;
    ff::LaunchShape shape{s->ppt, s->block, s->blocks_per_sm, s->num_sms};
    const bool fusable = image_is_device && s->rhs_id == FF_RHS_LORENZ && !s->tape_on && s->check_every == 0 &&
                         n_steps > 0 && s->n_particles > 0 && std::isfinite(dt) &&
                         ff::lorenz_uniform_packed(s->method, (s->flags & FF_FLAG_KAHAN) != 0,
                                                   s->pparam_index >= 0, probe, shape);
    if (!fusable) {
        st = ff_step(s, n_steps, dt);
        if (st != FF_OK) return st;
        const int64_t integrator_launches = s->last_integrator_launches;
        st = ff_project_splat(s, v, image, image_is_device);
        s->last_integrator_launches = integrator_launches;  // ff_project_splat counted only its own
        return st;
    }
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_step_splat: set device");
    if (!v->accumulate) {
        cudaError_t e = cudaMemsetAsync(image, 0, sizeof(uint32_t) * (size_t)v->width * v->height, s->stream);
        if (e != cudaSuccess) return cuda_fail(e, "ff_step_splat: image clear");
    }
    va.image = image;
    st = integrate_steps(s, n_steps, dt, &va);
    if (st != FF_OK) return st;
    ff::account_steps(s, n_steps, dt);
    return FF_OK;
}

ff_status ff_get_state(ff_system* s, float* dst, int dst_is_device) {
    if (!s || !dst) return fail(FF_ERR_INVALID_ARG, "ff_get_state: NULL argument");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_get_state: set device");
    if (s->n_particles == 0) return FF_OK;
    cudaError_t e = cudaMemcpy2DAsync(dst, sizeof(float) * s->n_particles, s->d_state, sizeof(float) * s->pitch,
                                      sizeof(float) * s->n_particles, s->dim,
                                      dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                      s->stream);
    if (e == cudaSuccess && !dst_is_device) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_get_state: copy");
    return FF_OK;
}

ff_status ff_set_state(ff_system* s, const float* src, int src_is_device) {
    if (!s || !src) return fail(FF_ERR_INVALID_ARG, "ff_set_state: NULL argument");
    if (s->n_particles < 1) return fail(FF_ERR_STATE, "ff_set_state: no particles seeded");
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_set_state: set device");
    cudaError_t e = cudaMemcpy2DAsync(s->d_state, sizeof(float) * s->pitch, src, sizeof(float) * s->n_particles,
                                      sizeof(float) * s->n_particles, s->dim,
                                      src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                      s->stream);
    if (e == cudaSuccess && s->d_comp)
        e = cudaMemsetAsync(s->d_comp, 0, sizeof(float) * (size_t)s->pitch * s->dim, s->stream);
    if (e == cudaSuccess && !src_is_device) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_set_state: copy");
    s->tape_on = false;
    return clear_reset_state(s);
}

ff_status ff_stats(ff_system* s, int64_t* n_escaped, double* t_fwd, double* t_bwd) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_stats: system is NULL");
    if (t_fwd) *t_fwd = s->t_fwd;
    if (t_bwd) *t_bwd = s->t_bwd;
    if (!n_escaped) return FF_OK;
    DeviceScope dev(s->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_stats: set device");
    cudaError_t e = ff::launch_escape_count(s->d_state, s->pitch, s->dim, s->n_particles, s->d_counter,
                                            s->num_sms, s->stream);
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, s->d_counter, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(e, "ff_stats: escape count");
    *n_escaped = (int64_t)h;
    return FF_OK;
}

ff_status ff_system_info(ff_system* s, int64_t* n_particles, int64_t* pitch, int* dim, int* n_groups) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_system_info: system is NULL");
    if (n_particles) *n_particles = s->n_particles;
    if (pitch) *pitch = s->pitch;
    if (dim) *dim = s->dim;
    if (n_groups) *n_groups = s->n_groups;
    return FF_OK;
}

ff_status ff_last_launch(ff_system* s, char* kernel, int kernel_len, int* grid, int* block, int* fused_splat,
                         int64_t* integrator_launches, int64_t* splat_launches) {
    if (!s) return fail(FF_ERR_INVALID_ARG, "ff_last_launch: system is NULL");
    if (kernel && kernel_len < 1) return fail(FF_ERR_INVALID_ARG, "ff_last_launch: kernel_len < 1");
    if (grid) *grid = s->last_integrator.grid;
    if (block) *block = s->last_integrator.block;
    if (fused_splat) *fused_splat = s->last_fused ? 1 : 0;
    if (integrator_launches) *integrator_launches = s->last_integrator_launches;
    if (splat_launches) *splat_launches = s->last_splat_launches;
    if (!kernel) return FF_OK;
    kernel[0] = '\0';
    if (!s->last_integrator.kernel) return FF_OK;
    const char* mangled = nullptr;
    cudaError_t e = cudaFuncGetName(&mangled, s->last_integrator.kernel);
    if (e != cudaSuccess || !mangled) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidValue : e, "ff_last_launch: kernel name");
    int rc = -1;
    char* plain = abi::__cxa_demangle(mangled, nullptr, nullptr, &rc);
    snprintf(kernel, (size_t)kernel_len, "%s", (rc == 0 && plain) ? plain : mangled);
    std::free(plain);
    return FF_OK;
}


}  // extern "C"

namespace ff {
// Lets entry points defined in other translation units report through ff_last_error().
void set_last_error_message(const char* msg) { g_last_error = msg; }

LaunchRecord& last_launch_record() {
    static thread_local LaunchRecord record;
    return record;
}

cudaError_t launch_integrate(int rhs_id, int method, bool kahan, bool pp, const IntegrateArgs& a,
                             const LaunchShape& shape, cudaStream_t stream) {
    switch (rhs_id) {
    case FF_RHS_LORENZ:
        if (kahan && lorenz_kahan_packed(method, pp, a, shape)) return launch_integrate_lorenz_kahan(pp, a, shape, stream);
        return launch_integrate_lorenz(method, kahan, pp, a, shape, stream);
    case FF_RHS_WILSON_COWAN: return launch_integrate_wc(method, kahan, pp, a, shape, stream);
    case FF_RHS_HH3: return launch_integrate_hh3(method, kahan, pp, a, shape, stream);
    case FF_RHS_LINEAR:
    case FF_RHS_HARMONIC: return launch_integrate_linear(rhs_id, method, kahan, pp, a, shape, stream);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace ff
