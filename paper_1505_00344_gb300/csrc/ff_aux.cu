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
        const uint64_t jg = (uint64_t)(a.first + j);  // index within the whole group
        for (int k = 0; k < a.dim; ++k) {
            const uint64_t r = splitmix64_at(a.seed, jg * (uint64_t)a.dim + (uint64_t)k + 1u);
            const double u = (double)(r >> 40) * (1.0 / 16777216.0);
            const double v = __dadd_rn(a.lo[k], __dmul_rn(a.width[k], u));
            a.x[k * a.pitch + a.start + j] = __double2float_rn(v);
        }
    }
}

// Per-particle parameter: lo + (hi - lo) * (i / (total - 1)) in double, to float, for
// particles i = first .. first + P - 1 of a linspace over `total` particles.
__global__ void linspace_kernel(float* out, int64_t P, double lo, double width, int64_t first, int64_t total) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < P; j += stride) {
        const int64_t i = first + j;
        const double frac = (total > 1) ? __ddiv_rn((double)i, (double)(total - 1)) : 0.0;
        out[j] = __double2float_rn(__dadd_rn(lo, __dmul_rn(width, frac)));
    }
}

// ---------------------------------------------------------------------------
// Projection + splat (paper Appendix A: vertex shader = Model-View map,
// geometry shader = projection to the screen, fragment shader + GL_ONE
// blending = add this particle's contribution to its pixel).  Every float
// operation is rounded on its own (explicit _rn intrinsics, no contraction)
// so the pixel decision is reproducible bit for bit.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool group_selected(const SplatArgs& a, int64_t i) {
    int g = 0;
#pragma unroll
    for (int q = 1; q < FF_MAX_GROUPS; ++q)
        if (q < a.n_groups && i >= a.gstart[q]) g = q;
    return (a.v.mask >> g) & 1u;
}

// Global mode: each thread projects 4 consecutive particles (one 16-byte load
// per plane) and adds one count per drawn particle with a fire-and-forget
// global reduction; the image is small enough to stay in L2.
template <int NDV, bool MASKED>
__global__ void __launch_bounds__(kSplatBlock) splat_global_kernel(const __grid_constant__ SplatArgs a) {
    const int64_t n4 = (a.n + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
        const int64_t i0 = 4 * t;
        const float4 u4 = __ldcs(reinterpret_cast<const float4*>(a.ax[0] + i0));
        const float4 v4 = __ldcs(reinterpret_cast<const float4*>(a.ax[1] + i0));
        float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (NDV == 3) w4 = __ldcs(reinterpret_cast<const float4*>(a.ax[2] + i0));
        const float u[4] = {u4.x, u4.y, u4.z, u4.w}, v[4] = {v4.x, v4.y, v4.z, v4.w},
                    w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = i0 + j;
            int col, row;
            if (i < a.n && (!MASKED || group_selected(a, i)) && pixel_of<NDV>(a.v, u[j], v[j], w[j], col, row))
                atomicAdd(&a.v.image[(int64_t)row * a.v.W + col], 1u);
        }
    }
}

// Shared mode, for views where consecutive particles land in a narrow strip of
// the image (a linspace parameter on one axis: the bifurcation diagram).
// Each block takes chunks of kSplatChunk consecutive particles, finds their
// bounding box, counts them in a shared-memory histogram when the box fits and
// flushes every touched bin with one global atomic; a chunk whose box does not
// fit adds its counts directly.
template <int NDV, bool MASKED>
__global__ void __launch_bounds__(kSplatBlock) splat_shared_kernel(const __grid_constant__ SplatArgs a) {
    __shared__ uint32_t bins[kSplatBins];
    __shared__ int box[4];  // min col, max col, min row, max row
    const int tid = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * kSplatChunk; base < a.n;
         base += (int64_t)gridDim.x * kSplatChunk) {
        if (tid == 0) { box[0] = INT32_MAX; box[1] = -1; box[2] = INT32_MAX; box[3] = -1; }
        __syncthreads();
        int cols[kSplatPerThread], rows[kSplatPerThread];
        int cmin = INT32_MAX, cmax = -1, rmin = INT32_MAX, rmax = -1;
#pragma unroll
        for (int q = 0; q < kSplatPerThread; ++q) {
            const int64_t i = base + (int64_t)q * kSplatBlock + tid;
            int col = -1, row = -1;
            if (i < a.n && (!MASKED || group_selected(a, i))) {
                const float w = NDV == 3 ? a.ax[2][i] : 0.0f;
                if (!pixel_of<NDV>(a.v, a.ax[0][i], a.ax[1][i], w, col, row)) col = -1;
            }
            cols[q] = col;
            rows[q] = row;
            if (col >= 0) {
                cmin = min(cmin, col); cmax = max(cmax, col);
                rmin = min(rmin, row); rmax = max(rmax, row);
            }
        }
        cmin = __reduce_min_sync(0xffffffffu, cmin);
        cmax = __reduce_max_sync(0xffffffffu, cmax);
        rmin = __reduce_min_sync(0xffffffffu, rmin);
        rmax = __reduce_max_sync(0xffffffffu, rmax);
        if ((tid & 31) == 0 && cmax >= 0) {
            atomicMin(&box[0], cmin); atomicMax(&box[1], cmax);
            atomicMin(&box[2], rmin); atomicMax(&box[3], rmax);
        }
        __syncthreads();
        const int bc0 = box[0], bc1 = box[1], br0 = box[2], br1 = box[3];
        if (bc1 >= 0) {
            const int bw = bc1 - bc0 + 1, bh = br1 - br0 + 1;
            if ((int64_t)bw * bh <= kSplatBins) {
                const int area = bw * bh;
                for (int b = tid; b < area; b += kSplatBlock) bins[b] = 0u;
                __syncthreads();
#pragma unroll
                for (int q = 0; q < kSplatPerThread; ++q)
                    if (cols[q] >= 0) atomicAdd(&bins[(rows[q] - br0) * bw + (cols[q] - bc0)], 1u);
                __syncthreads();
                for (int b = tid; b < area; b += kSplatBlock) {
                    const uint32_t v = bins[b];
                    if (v) {
                        const int r = b / bw;
                        atomicAdd(&a.v.image[(int64_t)(br0 + r) * a.v.W + bc0 + (b - r * bw)], v);
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < kSplatPerThread; ++q)
                    if (cols[q] >= 0) atomicAdd(&a.v.image[(int64_t)rows[q] * a.v.W + cols[q]], 1u);
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

cudaError_t launch_linspace(float* out, int64_t P, double lo, double hi, int64_t first, int64_t total, int num_sms,
                            cudaStream_t s) {
    if (P <= 0) return cudaSuccess;
    linspace_kernel<<<grid_for(P, 256, num_sms, 8), 256, 0, s>>>(out, P, lo, hi - lo, first, total);
    return cudaGetLastError();
}

cudaError_t launch_splat(const SplatArgs& a, int ndim_view, bool masked, bool strip, int num_sms,
                         cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (strip) {
        const int64_t chunks = (a.n + kSplatChunk - 1) / kSplatChunk;
        const int64_t cap = (int64_t)num_sms * 8;
        const int grid = (int)(chunks < cap ? chunks : cap);
        if (ndim_view == 2) {
            if (masked) splat_shared_kernel<2, true><<<grid, kSplatBlock, 0, s>>>(a);
            else splat_shared_kernel<2, false><<<grid, kSplatBlock, 0, s>>>(a);
        } else {
            if (masked) splat_shared_kernel<3, true><<<grid, kSplatBlock, 0, s>>>(a);
            else splat_shared_kernel<3, false><<<grid, kSplatBlock, 0, s>>>(a);
        }
        return cudaGetLastError();
    }
    const int grid = grid_for((a.n + 3) / 4, kSplatBlock, num_sms, 8);
    if (ndim_view == 2) {
        if (masked) splat_global_kernel<2, true><<<grid, kSplatBlock, 0, s>>>(a);
        else splat_global_kernel<2, false><<<grid, kSplatBlock, 0, s>>>(a);
    } else {
        if (masked) splat_global_kernel<3, true><<<grid, kSplatBlock, 0, s>>>(a);
        else splat_global_kernel<3, false><<<grid, kSplatBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// Soft sprites (paper Appendix A, geometry + fragment shaders with additive
// blending).  Each thread projects 4 consecutive particles (16-byte plane
// loads) and walks each sprite's bounding box; every pixel centre inside the
// disc q = d^2 / R^2 < 1 receives (1 - q)^2 times the group's colour with one
// fire-and-forget 16-byte vector reduction, so the four channels of a pixel
// travel together.  Coverage arithmetic rounds every operation on its own, so
// the set of touched pixels is reproducible bit for bit.
__device__ __forceinline__ void red_add_v4(float4* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

template <int NDV, bool MASKED>
__global__ void __launch_bounds__(kSplatBlock) sprite_kernel(const __grid_constant__ SpriteArgs a) {
    const int64_t n4 = (a.n + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float R = a.R, lo_c = -R - 1.0f, hi_c = a.v.Wf + R + 1.0f, hi_r = a.v.Hf + R + 1.0f;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4; t += stride) {
        const int64_t i0 = 4 * t;
        const float4 u4 = __ldcs(reinterpret_cast<const float4*>(a.ax[0] + i0));
        const float4 v4 = __ldcs(reinterpret_cast<const float4*>(a.ax[1] + i0));
        float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (NDV == 3) w4 = __ldcs(reinterpret_cast<const float4*>(a.ax[2] + i0));
        const float u[4] = {u4.x, u4.y, u4.z, u4.w}, v[4] = {v4.x, v4.y, v4.z, v4.w},
                    w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t i = i0 + j;
            if (i >= a.n) continue;
            int g = 0;
#pragma unroll
            for (int q = 1; q < FF_MAX_GROUPS; ++q)
                if (q < a.n_groups && i >= a.gstart[q]) g = q;
            if (MASKED && !((a.v.mask >> g) & 1u)) continue;
            float pc, pr;
            if (!sprite_centre<NDV>(a.v, u[j], v[j], w[j], pc, pr)) continue;
            // off-window (and non-finite) centres are rejected before any integer conversion
            if (!(pc > lo_c && pc < hi_c && pr > lo_c && pr < hi_r)) continue;
            const int c0 = max(0, (int)floorf(pc - R)), c1 = min(a.v.W - 1, (int)ceilf(pc + R));
            const int r0 = max(0, (int)floorf(pr - R)), r1 = min(a.v.H - 1, (int)ceilf(pr + R));
            const float4 col = a.colour[g];
            for (int row = r0; row <= r1; ++row) {
                const float dy = __fsub_rn(__fadd_rn((float)row, 0.5f), pr);
                const float dy2 = __fmul_rn(dy, dy);
                float4* line = a.image + (int64_t)row * a.v.W;
                for (int c = c0; c <= c1; ++c) {
                    const float dx = __fsub_rn(__fadd_rn((float)c, 0.5f), pc);
                    const float q = __fmul_rn(__fadd_rn(__fmul_rn(dx, dx), dy2), a.inv_r2);
                    if (q < 1.0f) {
                        const float om = 1.0f - q;
                        const float wgt = om * om;
                        red_add_v4(line + c, wgt * col.x, wgt * col.y, wgt * col.z, wgt * col.w);
                    }
                }
            }
        }
    }
}

cudaError_t launch_sprites(const SpriteArgs& a, int ndim_view, bool masked, int num_sms, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const int grid = grid_for((a.n + 3) / 4, kSplatBlock, num_sms, 8);
    if (ndim_view == 2) {
        if (masked) sprite_kernel<2, true><<<grid, kSplatBlock, 0, s>>>(a);
        else sprite_kernel<2, false><<<grid, kSplatBlock, 0, s>>>(a);
    } else {
        if (masked) sprite_kernel<3, true><<<grid, kSplatBlock, 0, s>>>(a);
        else sprite_kernel<3, false><<<grid, kSplatBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tiled sprites.  The same centre, bounding box and coverage arithmetic as
// sprite_kernel, so the covered pixels and their weights are the same; only
// the order of the FP32 sums differs.
// ---------------------------------------------------------------------------
int sprite_tiles(int W, int H) {
    return ((W + kSpriteTile - 1) / kSpriteTile) * ((H + kSpriteTile - 1) / kSpriteTile);
}

int64_t sprite_entries_bound(int64_t n, float radius) {
    // a bounding box spans at most 2R + 3 pixels, so at most ceil((2R + 3) / T) + 1 tiles per axis
    const int per_axis = (int)ceilf((2.0f * radius + 3.0f) / kSpriteTile) + 1;
    return n * per_axis * per_axis;
}

// Centre, group and the clipped pixel bounding box of particle i; false if it draws nothing.
template <int NDV, bool MASKED>
__device__ __forceinline__ bool sprite_box(const SpriteArgs& a, int64_t i, float& pc, float& pr, int& g, int& c0,
                                           int& c1, int& r0, int& r1) {
    g = 0;
#pragma unroll
    for (int q = 1; q < FF_MAX_GROUPS; ++q)
        if (q < a.n_groups && i >= a.gstart[q]) g = q;
    if (MASKED && !((a.v.mask >> g) & 1u)) return false;
    const float w = NDV == 3 ? a.ax[2][i] : 0.0f;
    if (!sprite_centre<NDV>(a.v, a.ax[0][i], a.ax[1][i], w, pc, pr)) return false;
    const float R = a.R;
    if (!(pc > -R - 1.0f && pc < a.v.Wf + R + 1.0f && pr > -R - 1.0f && pr < a.v.Hf + R + 1.0f)) return false;
    c0 = max(0, (int)floorf(pc - R));
    c1 = min(a.v.W - 1, (int)ceilf(pc + R));
    r0 = max(0, (int)floorf(pr - R));
    r1 = min(a.v.H - 1, (int)ceilf(pr + R));
    return c0 <= c1 && r0 <= r1;
}

// Pass 1: per-tile particle counts (block histograms in shared memory).
template <int NDV, bool MASKED>
__global__ void __launch_bounds__(kSplatBlock) sprite_count_kernel(const __grid_constant__ SpriteArgs a,
                                                                     uint32_t* count, int tiles_x, int n_tiles) {
    __shared__ uint32_t hist[kSpriteMaxTiles];
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) hist[t] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        float pc, pr;
        int g, c0, c1, r0, r1;
        if (!sprite_box<NDV, MASKED>(a, i, pc, pr, g, c0, c1, r0, r1)) continue;
        for (int ty = r0 / kSpriteTile; ty <= r1 / kSpriteTile; ++ty)
            for (int tx = c0 / kSpriteTile; tx <= c1 / kSpriteTile; ++tx) atomicAdd(&hist[ty * tiles_x + tx], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
        if (hist[t]) atomicAdd(&count[t], hist[t]);
}

// Pass 2 (one block): offsets = exclusive prefix sum of the counts, cursors =
// offsets, and chunk offsets = exclusive prefix sum of ceil(count / chunk): a
// tile's list is rendered in chunks of kSpriteChunk entries by any block.
constexpr uint32_t kSpriteChunk = 512;
__global__ void __launch_bounds__(1024) sprite_scan_kernel(const uint32_t* count, uint32_t* offset, uint32_t* cursor,
                                                           uint32_t* chunk_off, int n_tiles) {
    __shared__ uint32_t part[1024], cpart[1024];
    const int per = (n_tiles + blockDim.x - 1) / blockDim.x;
    const int t0 = threadIdx.x * per;
    uint32_t sum = 0, csum = 0;
    for (int t = t0; t < t0 + per && t < n_tiles; ++t) {
        sum += count[t];
        csum += (count[t] + kSpriteChunk - 1) / kSpriteChunk;
    }
    part[threadIdx.x] = sum;
    cpart[threadIdx.x] = csum;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {  // inclusive scans of the thread sums
        const uint32_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0u;
        const uint32_t cv = threadIdx.x >= (unsigned)off ? cpart[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        cpart[threadIdx.x] += cv;
        __syncthreads();
    }
    uint32_t run = part[threadIdx.x] - sum, crun = cpart[threadIdx.x] - csum;
    for (int t = t0; t < t0 + per && t < n_tiles; ++t) {
        offset[t] = run;
        cursor[t] = run;
        chunk_off[t] = crun;
        run += count[t];
        crun += (count[t] + kSpriteChunk - 1) / kSpriteChunk;
    }
    if (threadIdx.x == blockDim.x - 1) {
        offset[n_tiles] = part[threadIdx.x];
        chunk_off[n_tiles] = cpart[threadIdx.x];
    }
}

// Pass 3: the tile lists.  Each block counts its particles per tile again,
// reserves one range per touched tile, then writes each particle's index into
// its ranges.
template <int NDV, bool MASKED>
__global__ void __launch_bounds__(kSplatBlock) sprite_fill_kernel(const __grid_constant__ SpriteArgs a,
                                                                    uint32_t* cursor, uint32_t* entries,
                                                                    int tiles_x, int n_tiles, uint32_t cap) {
    __shared__ uint32_t slot[kSpriteMaxTiles];
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) slot[t] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        float pc, pr;
        int g, c0, c1, r0, r1;
        if (!sprite_box<NDV, MASKED>(a, i, pc, pr, g, c0, c1, r0, r1)) continue;
        for (int ty = r0 / kSpriteTile; ty <= r1 / kSpriteTile; ++ty)
            for (int tx = c0 / kSpriteTile; tx <= c1 / kSpriteTile; ++tx) atomicAdd(&slot[ty * tiles_x + tx], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
        if (slot[t]) slot[t] = atomicAdd(&cursor[t], slot[t]);  // the block's range starts here
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        float pc, pr;
        int g, c0, c1, r0, r1;
        if (!sprite_box<NDV, MASKED>(a, i, pc, pr, g, c0, c1, r0, r1)) continue;
        for (int ty = r0 / kSpriteTile; ty <= r1 / kSpriteTile; ++ty)
            for (int tx = c0 / kSpriteTile; tx <= c1 / kSpriteTile; ++tx) {
                const uint32_t at = atomicAdd(&slot[ty * tiles_x + tx], 1u);
                if (at < cap) entries[at] = (uint32_t)i;
            }
    }
}

// Pass 4: blocks take chunks of the tile lists round-robin; a chunk's fragments
// accumulate in a shared-memory copy of its tile, which is then added to the
// image with one 16-byte vector reduction per touched pixel (chunks of one tile
// may run at the same time).
template <int NDV, bool MASKED>
__global__ void __launch_bounds__(kSplatBlock) sprite_tile_kernel(const __grid_constant__ SpriteArgs a,
                                                                    const uint32_t* offset, const uint32_t* chunk_off,
                                                                    const uint32_t* entries, int tiles_x, int n_tiles) {
    __shared__ float4 acc[kSpriteTile * kSpriteTile];
    const uint32_t total = chunk_off[n_tiles];
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        // the tile of chunk c: the last t with chunk_off[t] <= c
        int lo = 0, hi = n_tiles - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (chunk_off[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const int tile = lo;
        const uint32_t e0 = offset[tile] + (c - chunk_off[tile]) * kSpriteChunk;
        const uint32_t e1 = min(e0 + kSpriteChunk, offset[tile + 1]);
        const int tx0 = (tile % tiles_x) * kSpriteTile, ty0 = (tile / tiles_x) * kSpriteTile;
        for (int p = threadIdx.x; p < kSpriteTile * kSpriteTile; p += blockDim.x) acc[p] = make_float4(0.f, 0.f, 0.f, 0.f);
        __syncthreads();
        float* accf = reinterpret_cast<float*>(acc);
        for (uint32_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            const int64_t i = entries[e];
            float pc, pr;
            int g, c0, c1, r0, r1;
            if (i >= a.n || !sprite_box<NDV, MASKED>(a, i, pc, pr, g, c0, c1, r0, r1)) continue;
            c0 = max(c0, tx0);
            c1 = min(c1, tx0 + kSpriteTile - 1);
            r0 = max(r0, ty0);
            r1 = min(r1, ty0 + kSpriteTile - 1);
            const float4 col = a.colour[g];
            for (int row = r0; row <= r1; ++row) {
                const float dy = __fsub_rn(__fadd_rn((float)row, 0.5f), pr);
                const float dy2 = __fmul_rn(dy, dy);
                for (int x = c0; x <= c1; ++x) {
                    const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), pc);
                    const float q = __fmul_rn(__fadd_rn(__fmul_rn(dx, dx), dy2), a.inv_r2);
                    if (q < 1.0f) {
                        const float om = 1.0f - q;
                        const float wgt = om * om;
                        float* px = accf + 4 * ((row - ty0) * kSpriteTile + (x - tx0));
                        atomicAdd(px + 0, wgt * col.x);
                        atomicAdd(px + 1, wgt * col.y);
                        atomicAdd(px + 2, wgt * col.z);
                        atomicAdd(px + 3, wgt * col.w);
                    }
                }
            }
        }
        __syncthreads();
        for (int p = threadIdx.x; p < kSpriteTile * kSpriteTile; p += blockDim.x) {
            const int row = ty0 + p / kSpriteTile, x = tx0 + p % kSpriteTile;
            const float4 t = acc[p];
            if (row < a.v.H && x < a.v.W && (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f))
                red_add_v4(a.image + (int64_t)row * a.v.W + x, t.x, t.y, t.z, t.w);
        }
        __syncthreads();
    }
}

template <int NDV, bool MASKED>
static cudaError_t tiled_passes(const SpriteArgs& a, uint32_t* tiles, uint32_t* entries, int num_sms,
                                cudaStream_t s) {
    const int tiles_x = (a.v.W + kSpriteTile - 1) / kSpriteTile;
    const int n_tiles = sprite_tiles(a.v.W, a.v.H);
    uint32_t* count = tiles;
    uint32_t* offset = tiles + n_tiles;             // n_tiles + 1 values
    uint32_t* cursor = tiles + 2 * n_tiles + 1;
    uint32_t* chunk_off = tiles + 3 * n_tiles + 1;  // n_tiles + 1 values
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(uint32_t) * n_tiles, s);
    if (e != cudaSuccess) return e;
    const int grid = grid_for(a.n, kSplatBlock, num_sms, 4);
    sprite_count_kernel<NDV, MASKED><<<grid, kSplatBlock, 0, s>>>(a, count, tiles_x, n_tiles);
    sprite_scan_kernel<<<1, 1024, 0, s>>>(count, offset, cursor, chunk_off, n_tiles);
    const uint32_t cap = (uint32_t)sprite_entries_bound(a.n, a.R);
    sprite_fill_kernel<NDV, MASKED><<<grid, kSplatBlock, 0, s>>>(a, cursor, entries, tiles_x, n_tiles, cap);
    sprite_tile_kernel<NDV, MASKED><<<num_sms * 8, kSplatBlock, 0, s>>>(a, offset, chunk_off, entries, tiles_x,
                                                                           n_tiles);
    return cudaGetLastError();
}

cudaError_t launch_sprites_tiled(const SpriteArgs& a, int ndim_view, bool masked, uint32_t* tiles,
                                 uint32_t* entries, int num_sms, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    if (ndim_view == 2)
        return masked ? tiled_passes<2, true>(a, tiles, entries, num_sms, s)
                      : tiled_passes<2, false>(a, tiles, entries, num_sms, s);
    return masked ? tiled_passes<3, true>(a, tiles, entries, num_sms, s)
                  : tiled_passes<3, false>(a, tiles, entries, num_sms, s);
}

cudaError_t launch_escape_count(const float* x, int64_t pitch, int dim, int64_t n,
                                unsigned long long* counter, int num_sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    escape_count_kernel<<<grid_for(n, 256, num_sms, 8), 256, 0, s>>>(x, pitch, dim, n, counter);
    return cudaGetLastError();
}

}  // namespace ff
