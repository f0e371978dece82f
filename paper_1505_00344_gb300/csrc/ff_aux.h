// ff_aux.h -- argument blocks and host launchers of the non-integrator kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ff.h"
#include "ff_project.cuh"

namespace ff {

struct SeedArgs {
    float* x;        // state planes
    int64_t pitch;
    int64_t start;   // first particle of the group
    int64_t count;
    int64_t first;   // index of the first of these particles within its whole group (a slice)
    uint64_t seed;
    int dim;
    int pad_;
    double lo[FF_MAX_DIM];
    double width[FF_MAX_DIM];  // hi - lo, formed in double on the host
};

constexpr int kSplatBlock = 256;
constexpr int kSplatPerThread = 16;
constexpr int kSplatChunk = kSplatBlock * kSplatPerThread;
constexpr int kSplatBins = 8192;  // 32 KB shared-memory histogram

struct SplatArgs {
    ViewArgs v;
    const float* ax[3];  // planes of the view axes (16-byte aligned; readable up to n rounded to 4)
    int64_t n;           // particles
    int n_groups;
    int64_t gstart[FF_MAX_GROUPS];
};

// Soft sprites: a square of half-side R pixels around each projected particle;
// pixel centres with q = d^2 / R^2 < 1 gain (1 - q)^2 times the group's colour.
struct SpriteArgs {
    ViewArgs v;            // projection (v.image unused)
    float4* image;         // [H][W] float4, channels interleaved, 16-byte aligned
    const float* ax[3];    // planes of the view axes (16-byte aligned; readable up to n rounded to 4)
    int64_t n;
    int n_groups;
    float R, inv_r2;       // radius and 1 / R^2 (formed in double, rounded)
    int64_t gstart[FF_MAX_GROUPS];
    float4 colour[FF_MAX_GROUPS];  // gain * colour per group
};

cudaError_t launch_seed(const SeedArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_sprites(const SpriteArgs& a, int ndim_view, bool masked, int num_sms, cudaStream_t s);

// Tiled sprites: particles are binned by the 32 x 32 pixel tiles their sprites
// touch, then blocks take chunks of the tile lists, accumulate each in shared memory and add
// it to the image.  Scratch: `tiles` holds 4 * n_tiles + 2 uint32 (counts,
// offsets, cursors, chunk offsets), `entries` the tile lists (sprite_entries_bound
// entries).
constexpr int kSpriteTile = 32;
constexpr int kSpriteMaxTiles = 8192;  // the shared-memory histograms' size
int sprite_tiles(int W, int H);          // tiles covering a W x H image
int64_t sprite_entries_bound(int64_t n, float radius);
cudaError_t launch_sprites_tiled(const SpriteArgs& a, int ndim_view, bool masked, uint32_t* tiles,
                                 uint32_t* entries, int num_sms, cudaStream_t s);
cudaError_t launch_linspace(float* out, int64_t P, double lo, double hi, int64_t first, int64_t total, int num_sms,
                            cudaStream_t s);
// strip: consecutive particles map to a narrow strip of the image (a linspace
// per-particle parameter on a view axis), so the shared-memory histogram pays.
cudaError_t launch_splat(const SplatArgs& a, int ndim_view, bool masked, bool strip, int num_sms,
                         cudaStream_t s);
cudaError_t launch_escape_count(const float* x, int64_t pitch, int dim, int64_t n,
                                unsigned long long* counter, int num_sms, cudaStream_t s);

}  // namespace ff
