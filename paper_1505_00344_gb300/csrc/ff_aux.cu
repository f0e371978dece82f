// ff_aux.cu -- the non-integrator kernels of the hot path: initial-condition
// seeding, per-particle parameter linspace, projection + point splat, and the
// escaped-particle count.
#include <cstdint>
#include <cuda_runtime.h>

#include "ff.h"
#include "ff_aux.h"

namespace ff {

// ---------------------------------------------------------------------------
// Seeding (paper Appendix A, "Particle Group" / "Initialization").
// SplitMix64 (Steele, Lea & Flood 2014): output n of the stream seeded with s
// is the variant-13 finaliser applied to s + n * 0x9E3779B97F4A7C15.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Group particle j, variable k: draw n = j*dim + k + 1; u = top 24 bits / 2^24;
// x = lo + width * u in double (separately rounded), then to nearest float.
__global__ void seed_kernel(const __grid_constant__ SeedArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < a.count; j += stride) {
        for (int k = 0; k < a.dim; ++k) {
            const uint64_t r = splitmix64_at(a.seed, (uint64_t)j * (uint64_t)a.dim + (uint64_t)k + 1u);
            const double u = (double)(r >> 40) * (1.0 / 16777216.0);
            const double v = __dadd_rn(a.lo[k], __dmul_rn(a.width[k], u));
            a.x[k * a.pitch + a.start + j] = __double2float_rn(v);
        }
    }
}

// Per-particle parameter: lo + (hi - lo) * (i / (P - 1)) in double, to float.
__global__ void linspace_kernel(float* out, int64_t P, double lo, double width) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
        const double frac = (P > 1) ? __ddiv_rn((double)i, (double)(P - 1)) : 0.0;
        out[i] = __double2float_rn(__dadd_rn(lo, __dmul_rn(width, frac)));
    }
}

// ---------------------------------------------------------------------------
// Projection + splat (paper Appendix A: vertex shader = Model-View map,
// geometry shader = projection to the screen, fragment shader + GL_ONE
// blending = add this particle's contribution to its pixel).  Every float
// operation is rounded on its own (explicit _rn intrinsics, no contraction)
// so the pixel decision is reproducible bit for bit.
// ---------------------------------------------------------------------------
template <int NDV>
__device__ __forceinline__ int pixel_of(const SplatArgs& a, int64_t i) {
    float fc, fr;
    if (NDV == 2) {
        const float u = a.ax[0][i], v = a.ax[1][i];
        fc = floorf(__fmul_rn(__fsub_rn(u, a.lo0), a.s0));
        fr = floorf(__fmul_rn(__fsub_rn(v, a.lo1), a.s1));
    } else {
        const float x = a.ax[0][i], y = a.ax[1][i], z = a.ax[2][i];
        float cl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float s = __fadd_rn(__fmul_rn(a.m[j], x), __fmul_rn(a.m[4 + j], y));
            s = __fadd_rn(s, __fmul_rn(a.m[8 + j], z));
            cl[j] = __fadd_rn(s, a.m[12 + j]);
        }
        if (!(cl[3] > 0.0f)) return -1;
        const float nx = __fdiv_rn(cl[0], cl[3]);
        const float ny = __fdiv_rn(cl[1], cl[3]);
        fc = floorf(__fmul_rn(__fsub_rn(nx, -1.0f), a.s0));
        fr = floorf(__fmul_rn(__fsub_rn(ny, -1.0f), a.s1));
    }
    if (!(fc >= 0.0f && fc < a.Wf && fr >= 0.0f && fr < a.Hf)) return -1;
    return (int)fr * a.W + (int)fc;
}

__device__ __forceinline__ bool group_selected(const SplatArgs& a, int64_t i) {
    int g = 0;
#pragma unroll
    for (int q = 1; q < FF_MAX_GROUPS; ++q)
        if (q < a.n_groups && i >= a.gstart[q]) g = q;
    return (a.mask >> g) & 1u;
}

// Each block takes chunks of kSplatChunk consecutive particles.  If the
// chunk's pixels fit a small bounding box (e.g. a bifurcation diagram, where
// consecutive particles share a parameter column) they are counted in a
// shared-memory histogram first and each touched bin is flushed with one
// global atomic; otherwise every warp merges equal pixels (match.any) and one
// lane per distinct pixel issues the global atomic.
template <int NDV, bool MASKED>
__global__ void __launch_bounds__(kSplatBlock) splat_kernel(const __grid_constant__ SplatArgs a) {
    __shared__ uint32_t bins[kSplatBins];
    __shared__ int box[4];  // min col, max col, min row, max row
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    for (int64_t base = (int64_t)blockIdx.x * kSplatChunk; base < a.n;
         base += (int64_t)gridDim.x * kSplatChunk) {
        if (tid == 0) { box[0] = INT32_MAX; box[1] = -1; box[2] = INT32_MAX; box[3] = -1; }
        __syncthreads();
        int pix[kSplatPerThread];
        int cmin = INT32_MAX, cmax = -1, rmin = INT32_MAX, rmax = -1;
#pragma unroll
        for (int q = 0; q < kSplatPerThread; ++q) {
            const int64_t i = base + (int64_t)q * kSplatBlock + tid;
            int p = -1;
            if (i < a.n && (!MASKED || group_selected(a, i))) p = pixel_of<NDV>(a, i);
            pix[q] = p;
            if (p >= 0) {
                const int r = p / a.W, c = p - r * a.W;
                cmin = min(cmin, c); cmax = max(cmax, c);
                rmin = min(rmin, r); rmax = max(rmax, r);
            }
        }
        cmin = __reduce_min_sync(0xffffffffu, cmin);
        cmax = __reduce_max_sync(0xffffffffu, cmax);
        rmin = __reduce_min_sync(0xffffffffu, rmin);
        rmax = __reduce_max_sync(0xffffffffu, rmax);
        if (lane == 0 && cmax >= 0) {
            atomicMin(&box[0], cmin); atomicMax(&box[1], cmax);
            atomicMin(&box[2], rmin); atomicMax(&box[3], rmax);
        }
        __syncthreads();
        const int bc0 = box[0], bc1 = box[1], br0 = box[2], br1 = box[3];
        if (bc1 < 0) {  // nothing drawn in this chunk
            __syncthreads();
            continue;
        }
        const int bw = bc1 - bc0 + 1, bh = br1 - br0 + 1;
        if ((int64_t)bw * bh <= kSplatBins) {
            const int area = bw * bh;
            for (int b = tid; b < area; b += kSplatBlock) bins[b] = 0u;
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kSplatPerThread; ++q) {
                const int p = pix[q];
                if (p >= 0) {
                    const int r = p / a.W, c = p - r * a.W;
                    atomicAdd(&bins[(r - br0) * bw + (c - bc0)], 1u);
                }
            }
            __syncthreads();
            for (int b = tid; b < area; b += kSplatBlock) {
                const uint32_t v = bins[b];
                if (v) {
                    const int r = br0 + b / bw, c = bc0 + b % bw;
                    atomicAdd(&a.image[(int64_t)r * a.W + c], v);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < kSplatPerThread; ++q) {
                const int p = pix[q];
                const unsigned drawn = __ballot_sync(0xffffffffu, p >= 0);
                if (p >= 0) {
                    const unsigned peers = __match_any_sync(drawn, p);
                    if (lane == __ffs(peers) - 1) atomicAdd(&a.image[p], (uint32_t)__popc(peers));
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Escaped particles: some component non-finite or above 1e30 in magnitude.
// One 64-bit counter (caller-provided device memory) per launch.
// ---------------------------------------------------------------------------
__global__ void escape_count_kernel(const float* x, int64_t pitch, int dim, int64_t n,
                                    unsigned long long* counter) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        bool esc = false;
        // compared in double (float -> double is exact), the same test as for FP64 states
        for (int k = 0; k < dim; ++k) esc |= !((double)fabsf(x[k * pitch + i]) <= 1e30);
        mine += esc ? 1ull : 0ull;
    }
    // warp sum, then one atomic per warp
    for (int off = 16; off > 0; off >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, off);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(counter, mine);
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static int grid_for(int64_t items, int block, int num_sms, int per_sm) {
    int64_t need = (items + block - 1) / block;
    int64_t cap = (int64_t)num_sms * per_sm;
    if (need > cap) need = cap;
    return need < 1 ? 1 : (int)need;
}

cudaError_t launch_seed(const SeedArgs& a, int num_sms, cudaStream_t s) {
    if (a.count <= 0) return cudaSuccess;
    seed_kernel<<<grid_for(a.count, 256, num_sms, 8), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_linspace(float* out, int64_t P, double lo, double hi, int num_sms,
                            cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    linspace_kernel<<<grid_for(P, 256, num_sms, 8), 256, 0, s>>>(out, P, lo, hi - lo);
    return cudaGetLastError();
}

cudaError_t launch_splat(const SplatArgs& a, int ndim_view, bool masked, int num_sms,
                         cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const int64_t chunks = (a.n + kSplatChunk - 1) / kSplatChunk;
    const int64_t cap = (int64_t)num_sms * 8;
    const int grid = (int)(chunks < cap ? chunks : cap);
    if (ndim_view == 2) {
        if (masked) splat_kernel<2, true><<<grid, kSplatBlock, 0, s>>>(a);
        else splat_kernel<2, false><<<grid, kSplatBlock, 0, s>>>(a);
    } else {
        if (masked) splat_kernel<3, true><<<grid, kSplatBlock, 0, s>>>(a);
        else splat_kernel<3, false><<<grid, kSplatBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_escape_count(const float* x, int64_t pitch, int dim, int64_t n,
                                unsigned long long* counter, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    escape_count_kernel<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(x, pitch, dim, n, counter);
    return cudaGetLastError();
}

}  // namespace ff
