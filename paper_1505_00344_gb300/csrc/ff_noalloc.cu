// ff_noalloc.cu -- escaped-particle counting that allocates no memory.
//
// ff_stats counts escaped particles with a counter that ff_create_system
// allocates.  Some callers cannot allocate device memory at the moment they
// want that count: a host application that hands a plugin its device buffers
// but owns the whole memory budget, a real-time render loop where cudaMalloc's
// implicit device synchronisation would stall the frame, or code whose memory
// all comes from a fixed pool sized up front.  ff_count_escaped_noalloc serves
// them: the caller passes the state (device) and receives the counts (host),
// and the only scratch -- one 64-bit counter per group -- is a fixed
// file-scope device array that exists on every GPU that loads the library
// until the process exits.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "ff.h"

namespace {

// Scratch: one counter per group.  Shared by every call on a device; the
// entry point clears the counters it uses before each launch.
static __device__ __align__(256) unsigned long long g_noalloc_counters[FF_NOALLOC_MAX_GROUPS];

struct CountArgs {
    const float* x;
    int64_t pitch;
    int64_t n;
    int dim;
    int n_groups;
    unsigned long long* counters;
    int64_t starts[FF_NOALLOC_MAX_GROUPS];
};

// Same escape test as the counter kernel behind ff_stats (some component not
// finite or above 1e30 in magnitude, compared in double); the count goes to the
// counter of the particle's group, merged per warp before the atomic.
__global__ void escape_count_groups_kernel(const __grid_constant__ CountArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // every lane of a warp runs the same number of iterations (warp-aligned bounds)
    const int64_t span = (a.n + 31) / 32 * 32;
    for (int64_t i = first; i < span; i += stride) {
        bool esc = false;
        int g = -1;
        if (i < a.n) {
            for (int k = 0; k < a.dim; ++k) esc |= !((double)fabsf(a.x[k * a.pitch + i]) <= 1e30);
            // last group whose start is <= i (starts are non-decreasing, starts[0] == 0)
            int lo = 0, hi = a.n_groups - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.starts[mid] <= i) lo = mid; else hi = mid - 1;
            }
            g = lo;
        }
        const int key = esc ? g : -1;
        const unsigned active = __ballot_sync(0xffffffffu, key >= 0);
        if (key >= 0) {
            const unsigned peers = __match_any_sync(active, key);
            if ((int)(threadIdx.x & 31) == __ffs(peers) - 1)
                atomicAdd(&a.counters[key], (unsigned long long)__popc(peers));
        }
    }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_lock;
void* g_scratch[64] = {};

ff_status scratch_for_current_device(void** out, int* dev_out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return FF_ERR_CUDA;
    if (dev < 0 || dev >= 64) return FF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_counters);
        if (e != cudaSuccess || !p) return FF_ERR_CUDA;
        g_scratch[dev] = p;
    }
    *out = g_scratch[dev];
    *dev_out = dev;
    return FF_OK;
}

}  // namespace

namespace ff {
void set_last_error_message(const char* msg);  // ff_api.cu: the text ff_last_error() returns
}

namespace {
ff_status fail(ff_status s, const char* msg) {
    ff::set_last_error_message(msg);
    return s;
}
}  // namespace

extern "C" ff_status ff_count_escaped_noalloc(const float* state_dev, int dim, int64_t n_particles,
                                              int64_t pitch, const int64_t* group_starts, int n_groups,
                                              void* cuda_stream, int64_t* counts_out) {
    if (!state_dev || !group_starts || !counts_out)
        return fail(FF_ERR_INVALID_ARG, "ff_count_escaped_noalloc: NULL argument");
    if (dim < 1 || dim > FF_MAX_DIM || n_particles < 0 || pitch < n_particles)
        return fail(FF_ERR_INVALID_ARG, "ff_count_escaped_noalloc: dim, n_particles or pitch out of range");
    if (n_groups < 1 || n_groups > FF_NOALLOC_MAX_GROUPS)
        return fail(FF_ERR_INVALID_ARG,
                    "ff_count_escaped_noalloc: n_groups must be 1..FF_NOALLOC_MAX_GROUPS (256)");
    if (group_starts[0] != 0) return fail(FF_ERR_INVALID_ARG, "ff_count_escaped_noalloc: group_starts[0] != 0");
    for (int g = 1; g < n_groups; ++g)
        if (group_starts[g] < group_starts[g - 1] || group_starts[g] > n_particles)
            return fail(FF_ERR_INVALID_ARG, "ff_count_escaped_noalloc: group_starts not non-decreasing in [0, n]");
    void* scratch = nullptr;
    int dev = 0;
    ff_status st = scratch_for_current_device(&scratch, &dev);
    if (st != FF_OK) return fail(st, "ff_count_escaped_noalloc: scratch address lookup failed");
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    CountArgs a{};
    a.x = state_dev;
    a.pitch = pitch;
    a.n = n_particles;
    a.dim = dim;
    a.n_groups = n_groups;
    a.counters = static_cast<unsigned long long*>(scratch);
    for (int g = 0; g < n_groups; ++g) a.starts[g] = group_starts[g];
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * n_groups, stream);
    if (e == cudaSuccess && n_particles > 0) {
        int sms = 1;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) {
            int64_t need = (n_particles + 255) / 256;
            const int64_t cap = (int64_t)sms * 8;
            const int grid = (int)(need < cap ? need : cap);
            escape_count_groups_kernel<<<grid, 256, 0, stream>>>(a);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts_out, scratch, sizeof(unsigned long long) * n_groups, cudaMemcpyDeviceToHost,
                            stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(FF_ERR_CUDA, "ff_count_escaped_noalloc: CUDA error");
    return FF_OK;
}
