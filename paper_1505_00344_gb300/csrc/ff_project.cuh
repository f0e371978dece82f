// ff_project.cuh -- the pixel rule of the render techniques (paper Appendix A:
// vertex shader = Model-View map, geometry shader = projection to the screen,
// fragment shader + GL_ONE blending = add this particle's count to its pixel),
// shared by the splat kernels and the integrator's fused splat epilogue.  Every
// float operation is rounded on its own (explicit _rn intrinsics, no
// contraction) so the pixel decision is reproducible bit for bit.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ff.h"

namespace ff {

struct ViewArgs {
    uint32_t* image;
    int W, H;
    float Wf, Hf;
    float lo0, s0, lo1, s1;  // 2D window (3D: lo = -1, s = W/2, H/2)
    float m[16];             // 3D Model-View-Projection, column-major
    int ndim;                // 2 or 3
    int axes[3];             // state variables (== dim: the per-particle parameter)
    uint32_t mask;           // groups drawn
};

// Pixel of one projected particle (col, row); false if it is not drawn.
template <int NDV>
__device__ __forceinline__ bool pixel_of(const ViewArgs& a, float u, float v, float w, int& col, int& row) {
    float fc, fr;
    if (NDV == 2) {
        fc = floorf(__fmul_rn(__fsub_rn(u, a.lo0), a.s0));
        fr = floorf(__fmul_rn(__fsub_rn(v, a.lo1), a.s1));
    } else {
        float cl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float t = __fadd_rn(__fmul_rn(a.m[j], u), __fmul_rn(a.m[4 + j], v));
            t = __fadd_rn(t, __fmul_rn(a.m[8 + j], w));
            cl[j] = __fadd_rn(t, a.m[12 + j]);
        }
        if (!(cl[3] > 0.0f)) return false;
        const float nx = __fdiv_rn(cl[0], cl[3]);
        const float ny = __fdiv_rn(cl[1], cl[3]);
        fc = floorf(__fmul_rn(__fsub_rn(nx, -1.0f), a.s0));
        fr = floorf(__fmul_rn(__fsub_rn(ny, -1.0f), a.s1));
    }
    if (!(fc >= 0.0f && fc < a.Wf && fr >= 0.0f && fr < a.Hf)) return false;
    col = (int)fc;
    row = (int)fr;
    return true;
}

// Continuous pixel coordinates of a projected particle (the pixel rule before
// its floor): the centre of its soft sprite.  False if it is behind the camera.
template <int NDV>
__device__ __forceinline__ bool sprite_centre(const ViewArgs& a, float u, float v, float w, float& pc, float& pr) {
    if constexpr (NDV == 2) {
        pc = __fmul_rn(__fsub_rn(u, a.lo0), a.s0);
        pr = __fmul_rn(__fsub_rn(v, a.lo1), a.s1);
        return true;
    } else {
        float cl[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float t = __fadd_rn(__fmul_rn(a.m[j], u), __fmul_rn(a.m[4 + j], v));
            t = __fadd_rn(t, __fmul_rn(a.m[8 + j], w));
            cl[j] = __fadd_rn(t, a.m[12 + j]);
        }
        if (!(cl[3] > 0.0f)) return false;
        pc = __fmul_rn(__fsub_rn(__fdiv_rn(cl[0], cl[3]), -1.0f), a.s0);
        pr = __fmul_rn(__fsub_rn(__fdiv_rn(cl[1], cl[3]), -1.0f), a.s1);
        return true;
    }
}

}  // namespace ff
