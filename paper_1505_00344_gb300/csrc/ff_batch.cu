// ff_batch.cu -- many systems stepped together (not part of the paper): one
// persistent launch per right-hand-side family over a table of work tiles, the
// families as parallel branches of one CUDA graph, and an autotuner for the
// launch shape of each family.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include <cuda_runtime.h>

#include "ff.h"
#include "ff_device.cuh"
#include "ff_internal.h"

namespace ff {

// Work items [first, first + count) of member system `sys` of a family.
struct BatchTile {
    int sys;
    int pad_;
    int64_t first;
    int64_t count;
};

struct BatchArgs {
    const IntegrateArgs* sys;  // per member: the argument block its own ff_step would use
    const BatchTile* tiles;
    int n_tiles;
    int n_steps;
    float* const* ckpt;  // taped runs: per member, where to store the state before the steps (or NULL)
};

// Each block takes tiles round-robin; a tile's system (and so its parameters,
// groups and step sizes) is the same for the whole block.  A family's members
// either all have a per-particle parameter (PP) or none has.
template <class R, int METHOD, bool PP, int PPT>
__global__ void __launch_bounds__(R::MAX_BLOCK, MinBlocks<R>::value) batch_kernel(const __grid_constant__ BatchArgs b) {
    for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
        const BatchTile T = b.tiles[tile];
        const IntegrateArgs& a = b.sys[T.sys];
        float* ck = b.ckpt ? b.ckpt[T.sys] : nullptr;
        for (int64_t t = T.first + threadIdx.x; t < T.first + T.count; t += blockDim.x) {
            if (ck) {  // checkpoint of a taped chunk: the state this launch starts from
                const int64_t i0 = t * PPT;
                for (int k = 0; k < a.dim; ++k) {
                    float v[PPT];
                    Vec<PPT>::load(a.x + k * a.pitch + i0, v);
                    Vec<PPT>::store(ck + k * a.pitch + i0, v);
                }
            }
            integrate_item<R, METHOD, false, PP, PPT, false, false>(a, t, b.n_steps);  // checkpoint written above
        }
    }
}

// HH3 RK4 at two particles per thread: all three neurons of a particle pair packed
// (hh3_rk4_x2_item, bit-identical to one particle per thread), under its own register bound.
template <bool PP>
__global__ void __launch_bounds__(HH3::MAX_BLOCK / 2, 3) batch_hh3_x2_kernel(const __grid_constant__ BatchArgs b) {
    for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
        const BatchTile T = b.tiles[tile];
        const IntegrateArgs& a = b.sys[T.sys];
        float* ck = b.ckpt ? b.ckpt[T.sys] : nullptr;
        for (int64_t t = T.first + threadIdx.x; t < T.first + T.count; t += blockDim.x) {
            if (ck) {  // checkpoint of a taped chunk: the state this launch starts from
                const int64_t i0 = t * 2;
                for (int k = 0; k < a.dim; ++k) {
                    float v[2];
                    Vec<2>::load(a.x + k * a.pitch + i0, v);
                    Vec<2>::store(ck + k * a.pitch + i0, v);
                }
            }
            hh3_rk4_x2_item<PP, false>(a, t, b.n_steps);  // checkpoint written above
        }
    }
}

template <class R, int METHOD, bool PP>
static const void* kernel_pp(int ppt) {
    if (ppt == 1) return (const void*)batch_kernel<R, METHOD, PP, 1>;
    if constexpr (R::DIM <= 4) {
        if (ppt == 2) return (const void*)batch_kernel<R, METHOD, PP, 2>;
        if (ppt == 4) return (const void*)batch_kernel<R, METHOD, PP, 4>;
    }
    if constexpr (std::is_same<R, HH3>::value && METHOD == FF_RK4) {
        if (ppt == 2) return (const void*)batch_hh3_x2_kernel<PP>;
    }
    return nullptr;
}

// The kernel of a launch shape; nullptr for particles-per-thread the family does not have.
template <class R, int METHOD>
static const void* kernel_for(int ppt, bool pp) {
    return pp ? kernel_pp<R, METHOD, true>(ppt) : kernel_pp<R, METHOD, false>(ppt);
}

static const void* family_kernel(int rhs_id, int method, int ppt, bool pp) {
    const bool rk4 = method == FF_RK4;
    switch (rhs_id) {
    case FF_RHS_LORENZ: return rk4 ? kernel_for<Lorenz, FF_RK4>(ppt, pp) : kernel_for<Lorenz, FF_EULER>(ppt, pp);
    case FF_RHS_WILSON_COWAN:
        return rk4 ? kernel_for<WilsonCowan, FF_RK4>(ppt, pp) : kernel_for<WilsonCowan, FF_EULER>(ppt, pp);
    case FF_RHS_HH3: return rk4 ? kernel_for<HH3, FF_RK4>(ppt, pp) : kernel_for<HH3, FF_EULER>(ppt, pp);
    case FF_RHS_HARMONIC:
        return rk4 ? kernel_for<Harmonic, FF_RK4>(ppt, pp) : kernel_for<Harmonic, FF_EULER>(ppt, pp);
    case FF_RHS_LINEAR: return rk4 ? kernel_for<Linear, FF_RK4>(ppt, pp) : kernel_for<Linear, FF_EULER>(ppt, pp);
    default: return nullptr;
    }
}

}  // namespace ff

using ff::cuda_fail;
using ff::DeviceScope;
using ff::fail;

struct ff_batch {
    struct Family {
        int rhs_id = 0, method = 0, dim = 0;
        bool pp = false;  // members have a per-particle parameter
        std::vector<int> members;  // indices into systems
        int ppt = 1, block = 256, grid = 1;
        int steps_per_launch = 0;  // 0: one launch per call; else launches of at most this many steps
        std::vector<ff::BatchTile> tiles;
        std::vector<ff::IntegrateArgs> h_sys;
        ff::IntegrateArgs* d_sys = nullptr;
        ff::BatchTile* d_tiles = nullptr;
        size_t tiles_cap = 0;
        cudaStream_t side = nullptr;
        cudaEvent_t done = nullptr;
        double tuned_rate = 0.0;  // particle-steps/s of the chosen shape, if tuned
        // taped runs: per member, the checkpoint slot the next launch writes (or NULL)
        std::vector<float*> h_ckpt;
        float** d_ckpt = nullptr;
        // batched adjoint
        std::vector<ff::AdjointArgs> h_adj;
        std::vector<ff::AdjTile> adj_tiles;
        std::vector<int> row0;
        std::vector<double> h_dp;
        ff::AdjointArgs* d_adj = nullptr;
        ff::AdjTile* d_adj_tiles = nullptr;
        int* d_row0 = nullptr;
        double* d_partial = nullptr;
        double* d_dp = nullptr;
        size_t adj_tiles_cap = 0;
        float* d_adj_scratch = nullptr;  // HH x 3 adjoint sweep: one chunk of stage points per thread
        size_t adj_scratch_floats = 0;
    };
    int device = 0, num_sms = 1;
    cudaStream_t user = nullptr;   // the caller's stream
    cudaStream_t cap = nullptr;    // internal stream the graph is captured on and launched from
    cudaEvent_t fork = nullptr, join = nullptr;
    std::vector<ff_system*> systems;
    std::vector<int64_t> n_particles;  // at creation
    std::vector<bool> has_pp;          // per-particle parameter at creation
    std::vector<Family> fams;
    cudaGraphExec_t exec = nullptr;
    int graph_steps = -1;
    bool graph_taped = false;
    bool taped = false;  // the members' tapes were started by ff_batch_tape_begin
};

namespace {

ff_status build_tiles(ff_batch* b, ff_batch::Family& f) {
    f.tiles.clear();
    const int64_t tile_items = (int64_t)f.block * 4;
    for (int m = 0; m < (int)f.members.size(); ++m) {
        const ff_system* s = b->systems[f.members[m]];
        const int64_t n_vec = ((s->n_particles + 3) / 4 * 4) / f.ppt;
        for (int64_t first = 0; first < n_vec; first += tile_items) {
            ff::BatchTile t{};
            t.sys = m;
            t.first = first;
            t.count = (n_vec - first < tile_items) ? n_vec - first : tile_items;
            f.tiles.push_back(t);
        }
    }
    const void* k = ff::family_kernel(f.rhs_id, f.method, f.ppt, f.pp);
    if (!k) return fail(FF_ERR_INVALID_ARG, "ff_batch: %d particles per thread not available for this system", f.ppt);
    cudaFuncAttributes attr;
    cudaError_t e = cudaFuncGetAttributes(&attr, k);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch: kernel attributes");
    if (f.block > attr.maxThreadsPerBlock) f.block = attr.maxThreadsPerBlock / 32 * 32;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, f.block, 0);
    if (e != cudaSuccess || occ < 1) return cuda_fail(e == cudaSuccess ? cudaErrorInvalidConfiguration : e,
                                                       "ff_batch: occupancy");
    const int64_t cap = (int64_t)occ * b->num_sms;
    f.grid = (int)((int64_t)f.tiles.size() < cap ? (int64_t)f.tiles.size() : cap);
    if (f.tiles.size() > f.tiles_cap) {
        cudaFree(f.d_tiles);
        f.d_tiles = nullptr;
        e = cudaMalloc(&f.d_tiles, sizeof(ff::BatchTile) * f.tiles.size());
        if (e != cudaSuccess) return cuda_fail(e, "ff_batch: tile table");
        f.tiles_cap = f.tiles.size();
    }
    e = cudaMemcpy(f.d_tiles, f.tiles.data(), sizeof(ff::BatchTile) * f.tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch: tile upload");
    return FF_OK;
}

// The argument blocks of the members for this step size, in the family's layout.
ff_status upload_args(ff_batch* b, ff_batch::Family& f, const double* dts) {
    for (int m = 0; m < (int)f.members.size(); ++m) {
        const int idx = f.members[m];
        ff::IntegrateArgs& a = f.h_sys[m];
        ff::fill_integrate_args(b->systems[idx], dts[idx], &a);
        a.n_vec = ((b->systems[idx]->n_particles + 3) / 4 * 4) / f.ppt;
    }
    cudaError_t e = cudaMemcpyAsync(f.d_sys, f.h_sys.data(), sizeof(ff::IntegrateArgs) * f.h_sys.size(),
                                    cudaMemcpyHostToDevice, b->user);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch: argument upload");
    return FF_OK;
}

cudaError_t launch_family(const ff_batch::Family& f, int n_steps, cudaStream_t st, bool taped = false) {
    ff::BatchArgs args{f.d_sys, f.d_tiles, (int)f.tiles.size(), n_steps, taped ? f.d_ckpt : nullptr};
    void* params[] = {&args};
    return cudaLaunchKernel(ff::family_kernel(f.rhs_id, f.method, f.ppt, f.pp), dim3(f.grid), dim3(f.block), params, 0, st);
}

// Capture the fork/join graph of all families for this step count.
ff_status capture(ff_batch* b, int n_steps, bool taped) {
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch: begin capture");
    cudaError_t err = cudaEventRecord(b->fork, b->cap);
    for (auto& f : b->fams) {
        if (err == cudaSuccess) err = cudaStreamWaitEvent(f.side, b->fork, 0);
        // the branch: launches of at most steps_per_launch steps; only the first of a taped
        // segment stores the checkpoints
        const int per = f.steps_per_launch > 0 ? f.steps_per_launch : n_steps;
        for (int done = 0; done < n_steps && err == cudaSuccess; done += per)
            err = launch_family(f, per < n_steps - done ? per : n_steps - done, f.side, taped && done == 0);
        if (err == cudaSuccess) err = cudaEventRecord(f.done, f.side);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(b->cap, f.done, 0);
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap, &graph);
    if (err != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(err != cudaSuccess ? err : e, "ff_batch: capture");
    }
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch: graph instantiate");
    b->graph_steps = n_steps;
    b->graph_taped = taped;
    return FF_OK;
}

// One graph launch of n_steps for every member (taped: the families' checkpoint
// tables were filled by the caller), ordered after and before the caller's stream.
ff_status run_graph(ff_batch* b, int64_t n_steps, const double* dt, bool taped) {
    for (auto& f : b->fams) {
        ff_status st = upload_args(b, f, dt);
        if (st != FF_OK) return st;
        if (taped) {
            cudaError_t e = cudaMemcpyAsync(f.d_ckpt, f.h_ckpt.data(), sizeof(float*) * f.h_ckpt.size(),
                                            cudaMemcpyHostToDevice, b->user);
            if (e != cudaSuccess) return cuda_fail(e, "ff_batch_step: checkpoint table upload");
        }
    }
    if (!b->exec || b->graph_steps != (int)n_steps || b->graph_taped != taped) {
        ff_status st = capture(b, (int)n_steps, taped);
        if (st != FF_OK) return st;
    }
    cudaError_t e = cudaEventRecord(b->join, b->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->cap);
    if (e == cudaSuccess) e = cudaEventRecord(b->join, b->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->user, b->join, 0);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch_step: graph launch");
    return FF_OK;
}

ff_status check_members(ff_batch* b) {
    for (size_t i = 0; i < b->systems.size(); ++i)
        if (b->systems[i]->n_particles != b->n_particles[i] || b->systems[i]->tape_on != b->taped ||
            b->systems[i]->check_every > 0 || (b->systems[i]->pparam_index >= 0) != b->has_pp[i])
            return fail(FF_ERR_STATE, "ff_batch: member %zu changed since the batch was created", i);
    return FF_OK;
}

void destroy_batch(ff_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto& f : b->fams) {
        cudaFree(f.d_sys);
        cudaFree(f.d_tiles);
        cudaFree(f.d_ckpt);
        cudaFree(f.d_adj);
        cudaFree(f.d_adj_tiles);
        cudaFree(f.d_row0);
        cudaFree(f.d_partial);
        cudaFree(f.d_dp);
        cudaFree(f.d_adj_scratch);
        if (f.side) cudaStreamDestroy(f.side);
        if (f.done) cudaEventDestroy(f.done);
    }
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    delete b;
}

}  // namespace

extern "C" {

ff_status ff_batch_create(ff_system* const* systems, int n_systems, void* cuda_stream, ff_batch** out) {
    if (!out) return fail(FF_ERR_INVALID_ARG, "ff_batch_create: out is NULL");
    *out = nullptr;
    if (!systems || n_systems < 1) return fail(FF_ERR_INVALID_ARG, "ff_batch_create: no systems");
    for (int i = 0; i < n_systems; ++i) {
        const ff_system* s = systems[i];
        if (!s) return fail(FF_ERR_INVALID_ARG, "ff_batch_create: system %d is NULL", i);
        if (s->device != systems[0]->device) return fail(FF_ERR_INVALID_ARG, "ff_batch_create: systems on different devices");
        if (s->flags & FF_FLAG_KAHAN) return fail(FF_ERR_UNSUPPORTED, "ff_batch_create: system %d uses Kahan", i);
        if (s->check_every > 0) return fail(FF_ERR_UNSUPPORTED, "ff_batch_create: system %d has particle reset on", i);
        if (s->tape_on) return fail(FF_ERR_UNSUPPORTED, "ff_batch_create: system %d is taped", i);
        if (s->n_particles < 1) return fail(FF_ERR_STATE, "ff_batch_create: system %d has no particles", i);
        for (int j = 0; j < i; ++j)
            if (systems[j] == s) return fail(FF_ERR_INVALID_ARG, "ff_batch_create: system %d listed twice", i);
    }
    DeviceScope dev(systems[0]->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_batch_create: set device");
    ff_batch* b = new (std::nothrow) ff_batch();
    if (!b) return fail(FF_ERR_OOM, "ff_batch_create: host allocation");
    b->device = systems[0]->device;
    b->num_sms = systems[0]->num_sms;
    b->user = static_cast<cudaStream_t>(cuda_stream);
    for (int i = 0; i < n_systems; ++i) {
        b->systems.push_back(systems[i]);
        b->n_particles.push_back(systems[i]->n_particles);
        b->has_pp.push_back(systems[i]->pparam_index >= 0);
        int fi = -1;
        const bool pp = systems[i]->pparam_index >= 0;
        for (int q = 0; q < (int)b->fams.size(); ++q)
            if (b->fams[q].rhs_id == systems[i]->rhs_id && b->fams[q].method == systems[i]->method &&
                b->fams[q].pp == pp)
                fi = q;
        if (fi < 0) {
            ff_batch::Family f;
            f.rhs_id = systems[i]->rhs_id;
            f.method = systems[i]->method;
            f.pp = pp;
            f.dim = systems[i]->dim;
            b->fams.push_back(f);
            fi = (int)b->fams.size() - 1;
        }
        b->fams[fi].members.push_back(i);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    for (auto& f : b->fams) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&f.side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f.done, cudaEventDisableTiming);
        f.h_sys.resize(f.members.size());
        f.h_ckpt.assign(f.members.size(), nullptr);
        if (e == cudaSuccess) e = cudaMalloc(&f.d_sys, sizeof(ff::IntegrateArgs) * f.members.size());
        if (e == cudaSuccess) e = cudaMalloc(&f.d_ckpt, sizeof(float*) * f.members.size());
    }
    if (e != cudaSuccess) {
        ff_status st = cuda_fail(e, "ff_batch_create: resources");
        destroy_batch(b);
        return st;
    }
    for (auto& f : b->fams) {
        ff_status st = build_tiles(b, f);
        if (st != FF_OK) {
            destroy_batch(b);
            return st;
        }
    }
    *out = b;
    return FF_OK;
}

ff_status ff_batch_destroy(ff_batch* b) {
    if (!b) return FF_OK;
    DeviceScope dev(b->device);
    cudaStreamSynchronize(b->cap);
    destroy_batch(b);
    return FF_OK;
}

ff_status ff_batch_step(ff_batch* b, int64_t n_steps, const double* dt) {
    if (!b) return fail(FF_ERR_INVALID_ARG, "ff_batch_step: batch is NULL");
    if (!dt) return fail(FF_ERR_INVALID_ARG, "ff_batch_step: dt is NULL");
    if (n_steps < 0 || n_steps > ((int64_t)1 << 30))
        return fail(FF_ERR_INVALID_ARG, "ff_batch_step: n_steps must be 0..2^30");
    for (size_t i = 0; i < b->systems.size(); ++i)
        if (!std::isfinite(dt[i])) return fail(FF_ERR_INVALID_ARG, "ff_batch_step: dt[%zu] not finite", i);
    ff_status st = check_members(b);
    if (st != FF_OK) return st;
    if (n_steps == 0) return FF_OK;
    DeviceScope dev(b->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_batch_step: set device");
    if (!b->taped) {
        st = run_graph(b, n_steps, dt, false);
        if (st != FF_OK) return st;
        for (size_t i = 0; i < b->systems.size(); ++i) {
            b->systems[i]->steps_total += n_steps;
            ff::account_steps(b->systems[i], n_steps, dt[i]);
        }
        return FF_OK;
    }
    // Taped: segments that end where any member's chunk ends (every checkpoint_every
    // steps, and where a member's parameters or dt changed); the first launch of a
    // member's chunk stores its checkpoint from the state it loads.
    int64_t left = n_steps;
    while (left > 0) {
        int64_t take = left;
        for (auto& f : b->fams) {
            for (size_t m = 0; m < f.members.size(); ++m) {
                const int idx = f.members[m];
                ff_system* s = b->systems[idx];
                const bool need_new = s->chunks.empty() || s->chunks.back().n_steps >= s->tape_every ||
                                      s->chunk_version != s->params_version || s->chunk_dt != dt[idx];
                f.h_ckpt[m] = nullptr;
                if (need_new) {
                    if ((int64_t)s->chunks.size() >= s->tape_slots)
                        return fail(FF_ERR_STATE, "ff_batch_step: member %d's tape is full", idx);
                    ff::AdjChunk c{};
                    c.n_steps = 0;
                    c.ckpt = (int)s->chunks.size();
                    for (int q = 0; q < s->n_params; ++q) c.p[ff::kernel_param_index(s, q)] = (float)s->params[q];
                    for (int g = 0; g < s->n_groups; ++g) c.gh[g] = (float)(s->groups[g].direction * dt[idx]);
                    s->chunks.push_back(c);
                    s->chunk_version = s->params_version;
                    s->chunk_dt = dt[idx];
                    f.h_ckpt[m] = s->d_ckpt + (int64_t)c.ckpt * s->dim * s->pitch;
                }
                const int64_t room = s->tape_every - s->chunks.back().n_steps;
                if (room < take) take = room;
            }
        }
        st = run_graph(b, take, dt, true);
        if (st != FF_OK) return st;
        for (size_t i = 0; i < b->systems.size(); ++i) {
            b->systems[i]->chunks.back().n_steps += (int)take;
            b->systems[i]->steps_total += take;
            ff::account_steps(b->systems[i], take, dt[i]);
        }
        left -= take;
    }
    return FF_OK;
}

ff_status ff_batch_tape_begin(ff_batch* b, int64_t checkpoint_every, int64_t max_steps) {
    if (!b) return fail(FF_ERR_INVALID_ARG, "ff_batch_tape_begin: batch is NULL");
    if (b->taped) return fail(FF_ERR_STATE, "ff_batch_tape_begin: already taped (ff_batch_tape_end first)");
    ff_status st = check_members(b);
    if (st != FF_OK) return st;
    DeviceScope dev(b->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_batch_tape_begin: set device");
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch_tape_begin: synchronise");
    for (size_t i = 0; i < b->systems.size(); ++i) {
        st = ff_tape_begin(b->systems[i], checkpoint_every, max_steps);
        if (st != FF_OK) {
            for (size_t j = 0; j < i; ++j) ff_tape_end(b->systems[j]);
            return st;
        }
    }
    b->taped = true;
    return FF_OK;
}

ff_status ff_batch_tape_end(ff_batch* b) {
    if (!b) return fail(FF_ERR_INVALID_ARG, "ff_batch_tape_end: batch is NULL");
    DeviceScope dev(b->device);
    cudaStreamSynchronize(b->user);
    for (auto* s : b->systems) ff_tape_end(s);
    b->taped = false;
    return FF_OK;
}

ff_status ff_batch_backward(ff_batch* b, const float* const* dL_dxT_dev, float* const* dL_dx0_dev,
                            double* dL_dp_host) {
    if (!b) return fail(FF_ERR_INVALID_ARG, "ff_batch_backward: batch is NULL");
    if (!dL_dxT_dev || !dL_dx0_dev || !dL_dp_host) return fail(FF_ERR_INVALID_ARG, "ff_batch_backward: NULL array");
    for (size_t i = 0; i < b->systems.size(); ++i)
        if (!dL_dxT_dev[i] || !dL_dx0_dev[i])
            return fail(FF_ERR_INVALID_ARG, "ff_batch_backward: NULL buffer of member %zu", i);
    if (!b->taped) return fail(FF_ERR_STATE, "ff_batch_backward: no tape (ff_batch_tape_begin before stepping)");
    ff_status st = check_members(b);
    if (st != FF_OK) return st;
    DeviceScope dev(b->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_batch_backward: set device");
    cudaError_t e = cudaSuccess;
    for (auto& f : b->fams) {
        const int nm = (int)f.members.size();
        f.h_adj.assign(nm, ff::AdjointArgs{});
        f.adj_tiles.clear();
        f.row0.assign(nm + 1, 0);
        for (int m = 0; m < nm && e == cudaSuccess; ++m) {
            const int idx = f.members[m];
            ff_system* s = b->systems[idx];
            if (!s->chunks.empty())
                e = cudaMemcpyAsync(s->d_chunks, s->chunks.data(), sizeof(ff::AdjChunk) * s->chunks.size(),
                                    cudaMemcpyHostToDevice, b->user);
            ff::AdjointArgs& a = f.h_adj[m];
            a.ckpt = s->d_ckpt;
            a.chunks = s->d_chunks;
            a.n_chunks = (int)s->chunks.size();
            a.dim = s->dim;
            a.lam_in = dL_dxT_dev[idx];
            a.lam_out = dL_dx0_dev[idx];
            a.pparam = s->d_pparam;
            a.pidx = s->pparam_index >= 0 ? ff::kernel_param_index(s, s->pparam_index) : -1;
            a.np_stride = FF_MAX_PARAMS;
            a.n = s->n_particles;
            a.pitch = s->pitch;
            a.n_groups = s->n_groups;
            a.max_chunk = (int)s->tape_every;
            for (int g = 0; g < s->n_groups; ++g) a.gstart[g] = s->groups[g].start;
            f.row0[m] = (int)f.adj_tiles.size();
            const int tile = ff::adjoint_tile_particles(f.rhs_id);
            for (int64_t first = 0; first < s->n_particles; first += tile) {
                ff::AdjTile t{};
                t.sys = m;
                t.first = first;
                t.count = s->n_particles - first < tile ? s->n_particles - first : tile;
                f.adj_tiles.push_back(t);
            }
        }
        f.row0[nm] = (int)f.adj_tiles.size();
        if (e != cudaSuccess) break;
        if (!f.d_adj) {
            e = cudaMalloc(&f.d_adj, sizeof(ff::AdjointArgs) * nm);
            if (e == cudaSuccess) e = cudaMalloc(&f.d_row0, sizeof(int) * (nm + 1));
            if (e == cudaSuccess) e = cudaMalloc(&f.d_dp, sizeof(double) * FF_MAX_PARAMS * nm);
        }
        if (e == cudaSuccess && f.adj_tiles.size() > f.adj_tiles_cap) {
            cudaFree(f.d_adj_tiles);
            cudaFree(f.d_partial);
            f.d_adj_tiles = nullptr;
            f.d_partial = nullptr;
            f.adj_tiles_cap = 0;
            e = cudaMalloc(&f.d_adj_tiles, sizeof(ff::AdjTile) * f.adj_tiles.size());
            if (e == cudaSuccess) e = cudaMalloc(&f.d_partial, sizeof(double) * FF_MAX_PARAMS * f.adj_tiles.size());
            if (e == cudaSuccess) f.adj_tiles_cap = f.adj_tiles.size();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(f.d_adj, f.h_adj.data(), sizeof(ff::AdjointArgs) * nm, cudaMemcpyHostToDevice, b->user);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(f.d_adj_tiles, f.adj_tiles.data(), sizeof(ff::AdjTile) * f.adj_tiles.size(),
                                cudaMemcpyHostToDevice, b->user);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(f.d_row0, f.row0.data(), sizeof(int) * (nm + 1), cudaMemcpyHostToDevice, b->user);
        if (e != cudaSuccess) break;
        ff::BatchAdjointArgs ba{f.d_adj, f.d_adj_tiles, (int)f.adj_tiles.size(), FF_MAX_PARAMS, f.d_partial};
        const ff_system* s0 = b->systems[f.members[0]];
        const int64_t scratch_threads = ff::adjoint_scratch_threads(f.rhs_id, f.method, f.pp, b->num_sms, true);
        if (scratch_threads > 0) {
            int64_t longest = 1;  // the longest chunk of any member
            for (int m = 0; m < nm; ++m) {
                const ff_system* s = b->systems[f.members[m]];
                if (s->tape_every > longest) longest = s->tape_every;
            }
            const size_t need = (size_t)scratch_threads * (size_t)longest *
                                (size_t)ff::adjoint_scratch_floats_per_step(f.rhs_id, f.method);
            if (need > f.adj_scratch_floats) {
                cudaFree(f.d_adj_scratch);  // waits for any sweep still reading it
                f.d_adj_scratch = nullptr;
                f.adj_scratch_floats = 0;
                e = cudaMalloc(&f.d_adj_scratch, sizeof(float) * need);
                if (e != cudaSuccess) break;
                f.adj_scratch_floats = need;
            }
            ba.scratch = f.d_adj_scratch;
            ba.scratch_threads = scratch_threads;
        }
        const int np_kernel = f.rhs_id == FF_RHS_LINEAR ? 64 : s0->n_params;
        e = ff::launch_batch_adjoint(f.rhs_id, f.method, f.pp, ff::adjoint_sub_steps(s0->tape_every), ba, f.d_row0,
                                     nm, np_kernel, b->num_sms, b->user, f.d_dp);
        if (e != cudaSuccess) break;
        f.h_dp.assign((size_t)FF_MAX_PARAMS * nm, 0.0);
        e = cudaMemcpyAsync(f.h_dp.data(), f.d_dp, sizeof(double) * FF_MAX_PARAMS * nm, cudaMemcpyDeviceToHost,
                            b->user);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch_backward");
    for (auto& f : b->fams)
        for (size_t m = 0; m < f.members.size(); ++m) {
            const int idx = f.members[m];
            const ff_system* s = b->systems[idx];
            for (int q = 0; q < FF_MAX_PARAMS; ++q)
                dL_dp_host[(size_t)idx * FF_MAX_PARAMS + q] =
                    q < s->n_params ? f.h_dp[m * FF_MAX_PARAMS + ff::kernel_param_index(s, q)] : 0.0;
        }
    return FF_OK;
}

ff_status ff_batch_autotune(ff_batch* b, const double* dt, int64_t trial_steps) {
    if (!b || !dt) return fail(FF_ERR_INVALID_ARG, "ff_batch_autotune: NULL argument");
    if (trial_steps < 1 || trial_steps > 100000) return fail(FF_ERR_INVALID_ARG, "ff_batch_autotune: trial_steps 1..1e5");
    ff_status st = check_members(b);
    if (st != FF_OK) return st;
    DeviceScope dev(b->device);
    if (dev.err != cudaSuccess) return cuda_fail(dev.err, "ff_batch_autotune: set device");
    cudaError_t e = cudaStreamSynchronize(b->user);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch_autotune: synchronise");
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch_autotune: events");
    st = FF_OK;
    for (auto& f : b->fams) {
        // snapshot the members' states: trials advance them, the snapshot puts them back
        std::vector<float*> saved(f.members.size(), nullptr);
        int64_t units = 0;
        for (size_t m = 0; m < f.members.size() && e == cudaSuccess; ++m) {
            const ff_system* s = b->systems[f.members[m]];
            const size_t bytes = sizeof(float) * (size_t)s->pitch * s->dim;
            e = cudaMalloc(&saved[m], bytes);
            if (e == cudaSuccess) e = cudaMemcpy(saved[m], s->d_state, bytes, cudaMemcpyDeviceToDevice);
            units += s->n_particles;
        }
        const int ppts[3] = {1, 2, 4};
        const int blocks[4] = {64, 128, 256, 512};
        double best = -1.0;
        int best_ppt = f.ppt, best_block = f.block;
        for (int pi = 0; pi < 3 && e == cudaSuccess && st == FF_OK; ++pi) {
            if (!ff::family_kernel(f.rhs_id, f.method, ppts[pi], f.pp)) continue;  // shape not built
            for (int bi = 0; bi < 4 && e == cudaSuccess && st == FF_OK; ++bi) {
                f.ppt = ppts[pi];
                f.block = blocks[bi];
                st = build_tiles(b, f);
                if (st != FF_OK) break;
                if (f.block != blocks[bi]) continue;  // clamped: the same shape as a smaller block
                st = upload_args(b, f, dt);
                if (st != FF_OK) break;
                e = launch_family(f, (int)trial_steps, b->user);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(t0, b->user);
                if (e == cudaSuccess) e = launch_family(f, (int)trial_steps, b->user);
                if (e == cudaSuccess) e = cudaEventRecord(t1, b->user);
                if (e == cudaSuccess) e = cudaEventSynchronize(t1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                const double rate = (double)units * trial_steps / (ms * 1e-3);
                if (e == cudaSuccess && rate > best) {
                    best = rate;
                    best_ppt = f.ppt;
                    best_block = f.block;
                }
            }
        }
        // steps per launch at the best shape: the whole call, or the trial split into 2 or 4 launches
        f.ppt = best_ppt;
        f.block = best_block;
        f.steps_per_launch = 0;
        if (st == FF_OK && e == cudaSuccess) st = build_tiles(b, f);
        if (st == FF_OK && e == cudaSuccess) st = upload_args(b, f, dt);
        for (int parts = 2; parts <= 4 && st == FF_OK && e == cudaSuccess && trial_steps >= parts; parts *= 2) {
            const int per = (int)((trial_steps + parts - 1) / parts);
            e = cudaEventRecord(t0, b->user);
            for (int64_t done = 0; done < trial_steps && e == cudaSuccess; done += per)
                e = launch_family(f, (int)(per < trial_steps - done ? per : trial_steps - done), b->user);
            if (e == cudaSuccess) e = cudaEventRecord(t1, b->user);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
            const double rate = (double)units * trial_steps / (ms * 1e-3);
            if (e == cudaSuccess && rate > best) {
                best = rate;
                f.steps_per_launch = per;
            }
        }
        // put the members' states back
        for (size_t m = 0; m < f.members.size(); ++m) {
            if (saved[m] && e == cudaSuccess) {
                const ff_system* s = b->systems[f.members[m]];
                e = cudaMemcpy(s->d_state, saved[m], sizeof(float) * (size_t)s->pitch * s->dim,
                               cudaMemcpyDeviceToDevice);
            }
            cudaFree(saved[m]);
        }
        f.tuned_rate = best;
        if (st != FF_OK || e != cudaSuccess) break;
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if (e != cudaSuccess) return cuda_fail(e, "ff_batch_autotune");
    return st;
}

ff_status ff_batch_describe(ff_batch* b, char* text, int text_len) {
    if (!b || !text || text_len < 1) return fail(FF_ERR_INVALID_ARG, "ff_batch_describe: NULL argument");
    static const char* names[] = {"linear", "harmonic", "wilson_cowan", "lorenz", "hh3"};
    std::string out;
    for (auto& f : b->fams) {
        char line[256];
        snprintf(line, sizeof(line), "%s/%s%s: %zu systems, %d particles/thread, block %d, grid %d, %zu tiles%s",
                 names[f.rhs_id], f.method == FF_RK4 ? "rk4" : "euler", f.pp ? "/per-particle" : "",
                 f.members.size(), f.ppt, f.block, f.grid, f.tiles.size(), f.tuned_rate > 0 ? "" : " (untuned)");
        out += line;
        if (f.steps_per_launch > 0) {
            snprintf(line, sizeof(line), ", at most %d steps per launch", f.steps_per_launch);
            out += line;
        }
        if (f.tuned_rate > 0) {
            snprintf(line, sizeof(line), ", tuned %.3e particle-steps/s", f.tuned_rate);
            out += line;
        }
        out += "\n";
    }
    snprintf(text, (size_t)text_len, "%s", out.c_str());
    return FF_OK;
}

}  // extern "C"
