// ff_peaks.cu -- issue-rate microbenchmark of the instruction kinds the
// integrators are built from (ff_pipe_rate in include/ff.h).
//
// The rooflines of the integrators are ALU rooflines: FP32 FMA for Lorenz, the
// multi-function unit (exp2, reciprocal) for Wilson-Cowan and the
// Hodgkin-Huxley rates.  Their peaks follow from unit counts and the SM clock,
// but the unit count of the multi-function pipe is not published per
// instruction, and a packed f32x2 FMA issues two lanes per instruction.  This
// kernel measures each rate on the device it runs on: every thread runs eight
// independent dependency chains of one instruction kind, at full occupancy on
// every SM, long enough (a few milliseconds) for the launch overhead to vanish.
#include <cstdint>

#include <cuda_runtime.h>

#include "ff.h"
#include "ff_device.cuh"

namespace ff {
void set_last_error_message(const char* msg);
}

namespace {

constexpr int kChains = 8;

// One step of a chain of instruction kind OP.  Every chain stays finite and
// bounded: FMA contracts towards a fixed point, ex2 of a negated value stays in
// [0.5, 1].  A chain of reciprocals alone would be an involution the compiler
// removes, so each reciprocal is followed by an FP32 add (a = 1/a + 0.001 stays
// near 1; the add runs on the FMA pipe beside it).  The logistic chain is the
// Wilson-Cowan sigmoid's own sequence, 1 / (1 + 2^-a): one ex2, one add, one
// reciprocal, so its rate shows how the two multi-function operations share
// the hardware.
template <int OP>
__device__ __forceinline__ float chain_step(float a) {
    if constexpr (OP == FF_PIPE_FFMA) return fmaf(a, 0.999999f, 1e-7f);
    else if constexpr (OP == FF_PIPE_EX2) return ff::ex2_ftz(-a);
    else if constexpr (OP == FF_PIPE_RCP) return __fadd_rn(ff::rcp_ftz(a), 0.001f);
    else return ff::rcp_ftz(__fadd_rn(1.0f, ff::ex2_ftz(-a)));
}

template <int OP>
__global__ void __launch_bounds__(256) pipe_kernel(float* out, int iters, float seed) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if constexpr (OP == FF_PIPE_FFMA2) {
        ff::f2 a[kChains];
        const ff::f2 m = ff::pack2(0.999999f, 0.999998f), c = ff::pack2(1e-7f, 2e-7f);
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = ff::pack2(seed + 0.01f * k, seed + 0.02f * tid);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = ff::fma2(a[k], m, c);
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            float x, y;
            ff::unpack2(a[k], x, y);
            s += x + y;
        }
        out[tid] = s;
    } else {
        float a[kChains];
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = seed + 0.01f * k + 1e-6f * (tid & 255);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = chain_step<OP>(a[k]);
        }
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kChains; ++k) s += a[k];
        out[tid] = s;
    }
}

template <int OP>
cudaError_t launch_pipe(float* out, int grid, int iters, cudaStream_t st) {
    pipe_kernel<OP><<<grid, 256, 0, st>>>(out, iters, 0.5f);
    return cudaGetLastError();
}

cudaError_t launch_op(int op, float* out, int grid, int iters, cudaStream_t st) {
    switch (op) {
    case FF_PIPE_FFMA: return launch_pipe<FF_PIPE_FFMA>(out, grid, iters, st);
    case FF_PIPE_FFMA2: return launch_pipe<FF_PIPE_FFMA2>(out, grid, iters, st);
    case FF_PIPE_EX2: return launch_pipe<FF_PIPE_EX2>(out, grid, iters, st);
    case FF_PIPE_RCP: return launch_pipe<FF_PIPE_RCP>(out, grid, iters, st);
    case FF_PIPE_LOGISTIC: return launch_pipe<FF_PIPE_LOGISTIC>(out, grid, iters, st);
    default: return cudaErrorInvalidValue;
    }
}

ff_status fail(ff_status s, const char* msg) {
    ff::set_last_error_message(msg);
    return s;
}

// Milliseconds of one timed launch of instruction kind op (after a warm-up launch).
cudaError_t time_op(int op, float* out, int grid, int iters, cudaStream_t st, cudaEvent_t t0, cudaEvent_t t1,
                    float* ms) {
    cudaError_t e = launch_op(op, out, grid, iters / 8, st);
    if (e == cudaSuccess) e = cudaEventRecord(t0, st);
    if (e == cudaSuccess) e = launch_op(op, out, grid, iters, st);
    if (e == cudaSuccess) e = cudaEventRecord(t1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, t0, t1);
    return e;
}

}  // namespace

extern "C" ff_status ff_pipe_rate(int op, int device, double* lane_ops_per_s) {
    if (!lane_ops_per_s) return fail(FF_ERR_INVALID_ARG, "ff_pipe_rate: NULL output");
    if (op < FF_PIPE_FFMA || op > FF_PIPE_LOGISTIC) return fail(FF_ERR_INVALID_ARG, "ff_pipe_rate: unknown op");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
    if (e != cudaSuccess) return fail(FF_ERR_CUDA, "ff_pipe_rate: set device");
    int sms = 1, per_sm = 1;
    float* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    float ms = 0.0f;
    const int iters = 4096;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pipe_kernel<FF_PIPE_FFMA2>, 256, 0);
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * (size_t)grid * 256);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    if (e == cudaSuccess) e = time_op(op, out, grid, iters, st, t0, t1, &ms);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (st) cudaStreamDestroy(st);
    if (out) cudaFree(out);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess || ms <= 0.0f) return fail(FF_ERR_CUDA, "ff_pipe_rate: measurement failed");
    // lane operations per chain step: two for a packed FMA, ex2 + rcp for the logistic
    const double lanes = (op == FF_PIPE_FFMA2 || op == FF_PIPE_LOGISTIC) ? 2.0 : 1.0;
    *lane_ops_per_s = (double)grid * 256.0 * kChains * (double)iters * lanes / (ms * 1e-3);
    return FF_OK;
}
