// ff_adjoint_impl.cuh -- device code and launch templates of the discrete
// adjoint of the RK4 / Euler integrator (not part of the paper), shared by the
// per-family translation units (ff_adjoint_lorenz.cu, ff_adjoint_hh3.cu,
// ff_adjoint_small.cu, ff_adjoint_linear.cu), which compile in parallel.
//
// One thread per particle walks the chunks in reverse with the adjoint state
// lambda = dL/dx in registers.  A chunk of L <= M*M steps is recomputed from its
// checkpoint twice (once when L <= M): once to place sub-checkpoints every M
// steps (local memory), then per sub-segment (in reverse) to put its <= M
// states in a shared-memory column per thread (the packed Lorenz sweep for
// chunks over 16 steps keeps its stage points there too), which the reverse
// RK4 steps consume from last to first.  Parameter gradients are summed
// per particle in FP32 within a chunk, added to FP64 per chunk, and reduced
// over particles through per-block FP64 partials in fixed order.  The
// 15-dimensional system runs a sweep of its own (ff_adjoint_hh3.cu: three lanes
// per particle pair, one recomputation per chunk into a global scratch).
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "ff.h"
#include "ff_adjoint.h"
#include "ff_device.cuh"

namespace ff {

// ---------------------------------------------------------------------------
// Vector-Jacobian products: jx = J(x)^T v and jp += F_p(x)^T v, differentiated
// by hand from the right-hand sides in ff_device.cuh.  No product is left for the
// compiler to fuse into a following addition (fmaf or _rn forms throughout), so
// every kernel that inlines them rounds the same way.
// ---------------------------------------------------------------------------
template <class R> struct Vjp;

template <> struct Vjp<Lorenz> {
    // f = (s (y - x), x (r - z) - y, x y - b z)
    __device__ __forceinline__ static void apply(const float (&x)[3], const float* p, const float (&v)[3],
                                                 float (&jx)[3], float* jp) {
        const float s = p[0], r = p[1], b = p[2];
        jx[0] = fmaf(-s, v[0], fmaf(r - x[2], v[1], x[1] * v[2]));
        jx[1] = fmaf(s, v[0], fmaf(x[0], v[2], -v[1]));
        jx[2] = fmaf(-x[0], v[1], -b * v[2]);
        jp[0] = fmaf(x[1] - x[0], v[0], jp[0]);
        jp[1] = fmaf(x[0], v[1], jp[1]);
        jp[2] = fmaf(-x[2], v[2], jp[2]);
    }
};

template <> struct Vjp<Harmonic> {
    // f = (v, -w^2 x)
    __device__ __forceinline__ static void apply(const float (&x)[2], const float* p, const float (&v)[2],
                                                 float (&jx)[2], float* jp) {
        const float w = p[0];
        jx[0] = -(w * w) * v[1];
        jx[1] = v[0];
        jp[0] = fmaf(-2.0f * w * x[0], v[1], jp[0]);
    }
};

template <> struct Vjp<WilsonCowan> {
    // f_E = (-E + S(aE)) / tauE, f_I = (-I + S(aI)) / tauI, S' = gain S (1 - S)
    __device__ __forceinline__ static void apply(const float (&x)[2], const float* p, const float (&v)[2],
                                                 float (&jx)[2], float* jp) {
        const float E = x[0], I = x[1];
        const float wEE = p[0], wEI = p[1], wIE = p[2], wII = p[3], tE = p[6], tI = p[7], g = p[8], th = p[9];
        const float aE = fmaf(wEE, E, fmaf(-wEI, I, p[4]));
        const float aI = fmaf(wIE, E, fmaf(-wII, I, p[5]));
        const float g2 = g * kLog2e;
        const float SE = rcp_ftz(1.0f + ex2_ftz(g2 * (th - aE)));
        const float SI = rcp_ftz(1.0f + ex2_ftz(g2 * (th - aI)));
        const float sE = SE * (1.0f - SE), sI = SI * (1.0f - SI);  // S'/gain
        const float uE = __fdividef(v[0], tE), uI = __fdividef(v[1], tI);  // v_k / tau_k
        const float dE = g * sE * uE, dI = g * sI * uI;                   // S'(a) v / tau
        jx[0] = fmaf(dI, wIE, fmaf(dE, wEE, -uE));
        jx[1] = fmaf(-dE, wEI, -fmaf(dI, wII, uI));
        jp[0] = fmaf(dE, E, jp[0]);
        jp[1] = fmaf(-dE, I, jp[1]);
        jp[2] = fmaf(dI, E, jp[2]);
        jp[3] = fmaf(-dI, I, jp[3]);
        jp[4] = __fadd_rn(jp[4], dE);
        jp[5] = __fadd_rn(jp[5], dI);
        jp[6] = fmaf(-(SE - E), __fdividef(uE, tE), jp[6]);   // d f_E / d tauE = -f_E / tauE
        jp[7] = fmaf(-(SI - I), __fdividef(uI, tI), jp[7]);
        jp[8] = fmaf(sE * (aE - th), uE, fmaf(sI * (aI - th), uI, jp[8]));
        jp[9] = __fsub_rn(__fsub_rn(jp[9], dE), dI);
    }
};

// d/dy of y / (1 - e^-y) by its series 1/2 + y/6 - y^3/180 + y^5/5040 - y^7/151200 (|y| < 0.5).
template <class O>
__device__ __forceinline__ typename O::T bernoulli_series_deriv_t(typename O::T y) {
    const auto y2 = O::mul(y, y);
    return O::fma(y, O::fma(y2, O::fma(y2, O::fma(y2, O::k(-1.0f / 151200.0f), O::k(1.0f / 5040.0f)),
                                       O::k(-1.0f / 180.0f)), O::k(1.0f / 6.0f)), O::k(0.5f));
}

template <> struct Vjp<Linear> {
    // f = A x (A padded to 8x8 row-major)
    __device__ __forceinline__ static void apply(const float (&x)[8], const float* p, const float (&v)[8],
                                                 float (&jx)[8], float* jp) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) s = fmaf(p[i * 8 + k], v[i], s);
            jx[k] = s;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int k = 0; k < 8; ++k) jp[i * 8 + k] = fmaf(v[i], x[k], jp[i * 8 + k]);
    }
};

// One forward step (plain FP32, unshifted) used by the recomputation.
// ---------------------------------------------------------------------------
// Lorenz RK4 in the shifted variable zt = z - r, the integrator's LorenzRK4Shift:
// the sweep keeps a chunk's states in (x, y, zt), so a recomputed step costs 37
// instead of 49 operations and a stage point 7 instead of 10.  The shift is a
// translation, so the Jacobian is the unshifted map's; it is evaluated with
// r - z = -zt and -z = -r - zt.  Every operation is explicit (no contraction),
// and the packed-pair sweep below repeats them lane by lane.
// ---------------------------------------------------------------------------
template <class R> struct IsLorenz { static constexpr bool value = false; };
template <> struct IsLorenz<Lorenz> { static constexpr bool value = true; };

struct LorenzShiftC {
    float s, ns, nb, nbr, nr, h1, h2, h6, nh1, nh2, nh6, sh1, sh2, sh6;
    __device__ __forceinline__ void init(float h, const float* p) {
        s = p[0];
        ns = -p[0];
        nb = -p[2];
        nbr = __fmul_rn(nb, p[1]);
        nr = -p[1];
        h1 = h;
        h2 = __fmul_rn(0.5f, h);
        h6 = __fmul_rn(h, 1.0f / 6.0f);
        nh1 = -h1;
        nh2 = -h2;
        nh6 = -h6;
        sh1 = __fmul_rn(s, h1);
        sh2 = __fmul_rn(s, h2);
        sh6 = __fmul_rn(s, h6);
    }
};

// One RK4 step of (x, y, zt): the operations of LorenzRK4Shift::acc and the plain update.
__device__ __forceinline__ void lorenz_shift_fwd(float (&x)[3], const LorenzShiftC& c) {
    float d, A, kz, X, Y, Z, a0, a1, a2;
    d = __fsub_rn(x[1], x[0]);
    A = fmaf(x[0], x[2], x[1]);
    kz = fmaf(x[0], x[1], fmaf(c.nb, x[2], c.nbr));
    a0 = d; a1 = A; a2 = kz;
    X = fmaf(c.sh2, d, x[0]); Y = fmaf(c.nh2, A, x[1]); Z = fmaf(c.h2, kz, x[2]);
    d = __fsub_rn(Y, X);
    A = fmaf(X, Z, Y);
    kz = fmaf(X, Y, fmaf(c.nb, Z, c.nbr));
    a0 = fmaf(2.0f, d, a0); a1 = fmaf(2.0f, A, a1); a2 = fmaf(2.0f, kz, a2);
    X = fmaf(c.sh2, d, x[0]); Y = fmaf(c.nh2, A, x[1]); Z = fmaf(c.h2, kz, x[2]);
    d = __fsub_rn(Y, X);
    A = fmaf(X, Z, Y);
    kz = fmaf(X, Y, fmaf(c.nb, Z, c.nbr));
    a0 = fmaf(2.0f, d, a0); a1 = fmaf(2.0f, A, a1); a2 = fmaf(2.0f, kz, a2);
    X = fmaf(c.sh1, d, x[0]); Y = fmaf(c.nh1, A, x[1]); Z = fmaf(c.h1, kz, x[2]);
    d = __fsub_rn(Y, X);
    A = fmaf(X, Z, Y);
    kz = fmaf(X, Y, fmaf(c.nb, Z, c.nbr));
    a0 = __fadd_rn(a0, d); a1 = __fadd_rn(a1, A); a2 = __fadd_rn(a2, kz);
    x[0] = fmaf(c.sh6, a0, x[0]); x[1] = fmaf(c.nh6, a1, x[1]); x[2] = fmaf(c.h6, a2, x[2]);
}

// The stage point x + c k(P) of the step from x, and d = y - x at P.
__device__ __forceinline__ void lorenz_shift_stage(const float (&P)[3], const float (&x)[3], float cs, float cn,
                                                   float ch, const LorenzShiftC& c, float (&out)[3], float& d) {
    d = __fsub_rn(P[1], P[0]);
    const float A = fmaf(P[0], P[2], P[1]);
    const float kz = fmaf(P[0], P[1], fmaf(c.nb, P[2], c.nbr));
    out[0] = fmaf(cs, d, x[0]);
    out[1] = fmaf(cn, A, x[1]);
    out[2] = fmaf(ch, kz, x[2]);
}

// jx = J^T v, jp += F_p^T v at the shifted point P with d = y - x there:
// J^T v = (-s v0 - zt v1 + y v2, s v0 - v1 + x v2, -x v1 - b v2),
// F_p^T v = ((y - x) v0, x v1, -z v2).
__device__ __forceinline__ void lorenz_shift_vjp(const float (&P)[3], float d, const LorenzShiftC& c,
                                                 const float (&v)[3], float (&jx)[3], float* jp) {
    const float nv1 = __fsub_rn(0.0f, v[1]);
    jx[0] = fmaf(c.ns, v[0], fmaf(P[2], nv1, __fmul_rn(P[1], v[2])));
    jx[1] = fmaf(c.s, v[0], fmaf(P[0], v[2], nv1));
    jx[2] = fmaf(P[0], nv1, __fmul_rn(c.nb, v[2]));
    jp[0] = fmaf(d, v[0], jp[0]);
    jp[1] = fmaf(P[0], v[1], jp[1]);
    jp[2] = fmaf(__fsub_rn(c.nr, P[2]), v[2], jp[2]);
}

// Reverse RK4 step from the shifted state x: the combination of adj_step below.
__device__ __forceinline__ void lorenz_shift_adj(const float (&x)[3], float (&lam)[3], const LorenzShiftC& c,
                                                 float* jp) {
    float x2[3], x3[3], x4[3], d1, d2, d3;
    lorenz_shift_stage(x, x, c.sh2, c.nh2, c.h2, c, x2, d1);
    lorenz_shift_stage(x2, x, c.sh2, c.nh2, c.h2, c, x3, d2);
    lorenz_shift_stage(x3, x, c.sh1, c.nh1, c.h1, c, x4, d3);
    const float d4 = __fsub_rn(x4[1], x4[0]);
    // u = h/6 lambda and 2u (= h/3 lambda rounded once) are the lambda terms of every l
    float u[3], u2[3], l[3], m[3], sum[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) { u[i] = __fmul_rn(c.h6, lam[i]); u2[i] = __fadd_rn(u[i], u[i]); }
    lorenz_shift_vjp(x4, d4, c, u, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = m[i]; l[i] = fmaf(c.h1, m[i], u2[i]); }
    lorenz_shift_vjp(x3, d3, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = __fadd_rn(sum[i], m[i]); l[i] = fmaf(c.h2, m[i], u2[i]); }
    lorenz_shift_vjp(x2, d2, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = __fadd_rn(sum[i], m[i]); l[i] = fmaf(c.h2, m[i], u[i]); }
    lorenz_shift_vjp(x, d1, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[i] = __fadd_rn(lam[i], __fadd_rn(sum[i], m[i]));
}

template <class R, int METHOD>
__device__ __forceinline__ void fwd_step(float (&x)[R::DIM], float h, const float* p) {
    constexpr int D = R::DIM;
    if (METHOD == FF_EULER) {
        float k[D];
        R::f(x, p, k);
#pragma unroll
        for (int i = 0; i < D; ++i) x[i] = fmaf(h, k[i], x[i]);
        return;
    }
    if constexpr (IsLorenz<R>::value) {
        LorenzShiftC c;
        c.init(h, p);
        lorenz_shift_fwd(x, c);
        return;
    } else if constexpr (!std::is_same<typename StepperFor<R, FF_RK4, false>::type, GenericRK4<R>>::value) {
        // the forward integrator's own RK4 stepper (HH3: the packed neuron pairs; Wilson-Cowan:
        // the shortened stage chain), so the recomputed states are the taped forward's, bit for bit
        typename StepperFor<R, FF_RK4, false>::type st;
        float acc[D], sc[D];
        st.init(h, p);
        st.acc(x, acc, sc);
#pragma unroll
        for (int i = 0; i < D; ++i) x[i] = fmaf(sc[i], acc[i], x[i]);
        return;
    }
    const float h2 = 0.5f * h, h6 = h * (1.0f / 6.0f);
    float k[D], xs[D], acc[D];
    R::f(x, p, k);
#pragma unroll
    for (int i = 0; i < D; ++i) { acc[i] = k[i]; xs[i] = fmaf(h2, k[i], x[i]); }
    R::f(xs, p, k);
#pragma unroll
    for (int i = 0; i < D; ++i) { acc[i] = fmaf(2.0f, k[i], acc[i]); xs[i] = fmaf(h2, k[i], x[i]); }
    R::f(xs, p, k);
#pragma unroll
    for (int i = 0; i < D; ++i) { acc[i] = fmaf(2.0f, k[i], acc[i]); xs[i] = fmaf(h, k[i], x[i]); }
    R::f(xs, p, k);
#pragma unroll
    for (int i = 0; i < D; ++i) x[i] = fmaf(h6, acc[i] + k[i], x[i]);
}

// Wilson-Cowan's reverse RK4 step.  The stage points are those of WilsonCowan::f
// (x2 = x + h/2 k1, x3 = x + h/2 k2, x4 = x + h k3), and the two logistic values of
// each stage point are kept from its evaluation (and formed once at x4), so the four
// products below need no exponential, reciprocal or division: 16 multi-function
// operations per reverse step instead of 12 for the stage points and 8 or more per
// product.  With S' = gain S (1 - S), u = v / tau and d = S'(a) u:
//   jx_E = wEE d_E + wIE d_I - u_E,   jx_I = -wEI d_E - wII d_I - u_I,
// and the parameter terms of Vjp<WilsonCowan>.
__device__ __forceinline__ void wc_vjp_given(float E, float I, float SE, float SI, const float* p, float iE, float iI,
                                             const float (&v)[2], float (&jx)[2], float* jp) {
    const float wEE = p[0], wEI = p[1], wIE = p[2], wII = p[3], g = p[8], th = p[9];
    const float aE = fmaf(wEE, E, fmaf(-wEI, I, p[4]));
    const float aI = fmaf(wIE, E, fmaf(-wII, I, p[5]));
    const float sE = SE * (1.0f - SE), sI = SI * (1.0f - SI);  // S'/gain
    const float uE = v[0] * iE, uI = v[1] * iI;                 // v_k / tau_k
    const float dE = g * sE * uE, dI = g * sI * uI;             // S'(a) v / tau
    jx[0] = fmaf(dI, wIE, fmaf(dE, wEE, -uE));
    jx[1] = fmaf(-dE, wEI, -fmaf(dI, wII, uI));
    jp[0] = fmaf(dE, E, jp[0]);
    jp[1] = fmaf(-dE, I, jp[1]);
    jp[2] = fmaf(dI, E, jp[2]);
    jp[3] = fmaf(-dI, I, jp[3]);
    jp[4] = __fadd_rn(jp[4], dE);
    jp[5] = __fadd_rn(jp[5], dI);
    jp[6] = fmaf(-(SE - E), uE * iE, jp[6]);  // d f_E / d tauE = -f_E / tauE
    jp[7] = fmaf(-(SI - I), uI * iI, jp[7]);
    jp[8] = fmaf(sE * (aE - th), uE, fmaf(sI * (aI - th), uI, jp[8]));
    jp[9] = __fsub_rn(__fsub_rn(jp[9], dE), dI);
}

__device__ __forceinline__ void wc_adj_step(const float (&x)[2], float (&lam)[2], float h, const float* p,
                                            float* jp) {
    const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
    // the right-hand side's constants, formed as WilsonCowan::f forms them
    const float g2 = p[8] * kLog2e;
    const float aEE = -g2 * p[0], aEI = g2 * p[1], cE = g2 * (p[9] - p[4]);
    const float aIE = -g2 * p[2], aII = g2 * p[3], cI = g2 * (p[9] - p[5]);
    const float iE = __fdividef(1.0f, p[6]), iI = __fdividef(1.0f, p[7]);
    float X[4][2], S[4][2];
    X[0][0] = x[0];
    X[0][1] = x[1];
#pragma unroll
    for (int st = 0; st < 4; ++st) {
        const float E = X[st][0], I = X[st][1];
        S[st][0] = rcp_ftz(1.0f + ex2_ftz(fmaf(aEE, E, fmaf(aEI, I, cE))));
        S[st][1] = rcp_ftz(1.0f + ex2_ftz(fmaf(aIE, E, fmaf(aII, I, cI))));
        if (st < 3) {
            const float c = (st == 2) ? h : h2;
            X[st + 1][0] = fmaf(c, fmaf(S[st][0], iE, -E * iE), x[0]);
            X[st + 1][1] = fmaf(c, fmaf(S[st][1], iI, -I * iI), x[1]);
        }
    }
    float l[2], m[2], sum[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) l[i] = h6 * lam[i];
    wc_vjp_given(X[3][0], X[3][1], S[3][0], S[3][1], p, iE, iI, l, m, jp);
#pragma unroll
    for (int i = 0; i < 2; ++i) { sum[i] = m[i]; l[i] = fmaf(h3, lam[i], h * m[i]); }
    wc_vjp_given(X[2][0], X[2][1], S[2][0], S[2][1], p, iE, iI, l, m, jp);
#pragma unroll
    for (int i = 0; i < 2; ++i) { sum[i] = __fadd_rn(sum[i], m[i]); l[i] = fmaf(h3, lam[i], h2 * m[i]); }
    wc_vjp_given(X[1][0], X[1][1], S[1][0], S[1][1], p, iE, iI, l, m, jp);
#pragma unroll
    for (int i = 0; i < 2; ++i) { sum[i] = __fadd_rn(sum[i], m[i]); l[i] = fmaf(h6, lam[i], h2 * m[i]); }
    wc_vjp_given(X[0][0], X[0][1], S[0][0], S[0][1], p, iE, iI, l, m, jp);
#pragma unroll
    for (int i = 0; i < 2; ++i) lam[i] = __fadd_rn(lam[i], __fadd_rn(sum[i], m[i]));
}

// Reverse of one step at state x: lambda <- (d step / d x)^T lambda, and the
// parameter contributions added to jp.  RK4 with stages x1 = x, x2 = x + h/2 k1,
// x3 = x + h/2 k2, x4 = x + h k3 and x' = x + h/6 (k1 + 2 k2 + 2 k3 + k4):
//   l4 = h/6 lam,           m4 = J(x4)^T l4
//   l3 = h/3 lam + h m4,    m3 = J(x3)^T l3
//   l2 = h/3 lam + h/2 m3,  m2 = J(x2)^T l2
//   l1 = h/6 lam + h/2 m2,  m1 = J(x1)^T l1
//   lam <- lam + m1 + m2 + m3 + m4,  jp += sum_s F_p(x_s)^T l_s.
template <class R, int METHOD>
__device__ __forceinline__ void adj_step(const float (&x)[R::DIM], float (&lam)[R::DIM], float h, const float* p,
                                         float* jp) {
    constexpr int D = R::DIM;
    if (METHOD == FF_EULER) {
        float l[D], m[D];
#pragma unroll
        for (int i = 0; i < D; ++i) l[i] = h * lam[i];
        Vjp<R>::apply(x, p, l, m, jp);
#pragma unroll
        for (int i = 0; i < D; ++i) lam[i] = __fadd_rn(lam[i], m[i]);
        return;
    }
    if constexpr (IsLorenz<R>::value) {
        LorenzShiftC c;
        c.init(h, p);
        lorenz_shift_adj(x, lam, c, jp);
        return;
    } else if constexpr (std::is_same<R, WilsonCowan>::value) {
        wc_adj_step(x, lam, h, p, jp);
        return;
    }
    const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
    static_assert(METHOD == FF_EULER || D <= 8, "the 15-dimensional system has a sweep of its own (ff_adjoint_hh3.cu)");
    float k[D], x2[D], x3[D], x4[D];
    R::f(x, p, k);
#pragma unroll
    for (int i = 0; i < D; ++i) x2[i] = fmaf(h2, k[i], x[i]);
    R::f(x2, p, k);
#pragma unroll
    for (int i = 0; i < D; ++i) x3[i] = fmaf(h2, k[i], x[i]);
    R::f(x3, p, k);
#pragma unroll
    for (int i = 0; i < D; ++i) x4[i] = fmaf(h, k[i], x[i]);
    float l[D], m[D], sum[D];
#pragma unroll
    for (int i = 0; i < D; ++i) l[i] = h6 * lam[i];
    Vjp<R>::apply(x4, p, l, m, jp);
#pragma unroll
    for (int i = 0; i < D; ++i) { sum[i] = m[i]; l[i] = fmaf(h3, lam[i], h * m[i]); }
    Vjp<R>::apply(x3, p, l, m, jp);
#pragma unroll
    for (int i = 0; i < D; ++i) { sum[i] = __fadd_rn(sum[i], m[i]); l[i] = fmaf(h3, lam[i], h2 * m[i]); }
    Vjp<R>::apply(x2, p, l, m, jp);
#pragma unroll
    for (int i = 0; i < D; ++i) { sum[i] = __fadd_rn(sum[i], m[i]); l[i] = fmaf(h6, lam[i], h2 * m[i]); }
    Vjp<R>::apply(x, p, l, m, jp);
#pragma unroll
    for (int i = 0; i < D; ++i) lam[i] = __fadd_rn(lam[i], __fadd_rn(sum[i], m[i]));
}

// Shared memory of a sweep's block: the sub-segment's M states of every thread (one column
// per thread, M * D floats; up to 64 KB for 128 threads of the 8-dimensional system).
template <class R, int M>
constexpr size_t sweep_smem(int block) { return sizeof(float) * M * R::DIM * (size_t)block; }

// Lets a kernel take more than the default 48 KB of dynamic shared memory where it needs to.
template <class Kernel>
static cudaError_t allow_smem(Kernel kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Reverse sweep of one particle i over all chunks: lambda from lam_in to
// lam_out, parameter contributions added to gacc (FP64, per chunk).  For systems
// of up to 8 dimensions (the 15-dimensional one has a sweep of its own).
template <class R, int METHOD, bool PP, int M>
__device__ __forceinline__ void adjoint_particle(const AdjointArgs& a, int64_t i, double (&gacc)[R::NP],
                                                 float* sts, int bs) {
    constexpr int D = R::DIM, NP = R::NP;
    int g = 0;
#pragma unroll
    for (int q = 1; q < FF_MAX_GROUPS; ++q)
        if (q < a.n_groups && i >= a.gstart[q]) g = q;
    float lam[D];
#pragma unroll
    for (int k = 0; k < D; ++k) lam[k] = (k < a.dim) ? a.lam_in[k * a.n + i] : 0.0f;
    const float pv = PP ? a.pparam[i] : 0.0f;
    for (int c = a.n_chunks - 1; c >= 0; --c) {
        const AdjChunk& ch = a.chunks[c];
        float p[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) p[q] = (PP && q == a.pidx) ? pv : ch.p[q];
        const float h = ch.gh[g];
        const int L = ch.n_steps;
        const float* ck = a.ckpt + (int64_t)ch.ckpt * a.dim * a.pitch;
        float x[D];
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = (k < a.dim) ? ck[k * a.pitch + i] : 0.0f;
        if constexpr (IsLorenz<R>::value && METHOD == FF_RK4) x[2] = __fsub_rn(x[2], p[1]);  // zt = z - r
        // sub-checkpoints every M steps (nothing to advance past the last one: a chunk of at
        // most M steps is recomputed once, by its only sub-segment)
        float cp[M][D];
        int nsub = 0;
        for (int base = 0; base < L; base += M, ++nsub) {
#pragma unroll
            for (int k = 0; k < D; ++k) cp[nsub][k] = x[k];
            const int nq = (base + M < L) ? M : 0;
#pragma unroll 1
            for (int r = 0; r < nq; ++r) fwd_step<R, METHOD>(x, h, p);
        }
        float jp[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) jp[q] = 0.0f;
        for (int sq = nsub - 1; sq >= 0; --sq) {
            const int nq = min(M, L - sq * M);
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = cp[sq][k];
            // the sub-segment's states in the thread's shared-memory column (state r,
            // component k at sts[(r * D + k) * bs]): the step loops stay rolled, so the
            // kernel keeps one copy of each step in the instruction cache (a register array
            // would need them unrolled M times)
#pragma unroll 2
            for (int r = 0; r < nq; ++r) {
#pragma unroll
                for (int k = 0; k < D; ++k) sts[(r * D + k) * bs] = x[k];
                if (r + 1 < nq) fwd_step<R, METHOD>(x, h, p);
            }
#pragma unroll 2
            for (int r = nq - 1; r >= 0; --r) {
                float xr[D];
#pragma unroll
                for (int k = 0; k < D; ++k) xr[k] = sts[(r * D + k) * bs];
                adj_step<R, METHOD>(xr, lam, h, p, jp);
            }
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) gacc[q] += (double)jp[q];
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
        if (k < a.dim) a.lam_out[k * a.n + i] = lam[k];
}

// Sum of gacc over the block into `row` (np_stride doubles), in a fixed order:
// warps by shuffles, then warp results in warp order.  Every thread of the
// block must call it.
template <int NP, int NW>
__device__ __forceinline__ void block_sum_to_row(double (&gacc)[NP], double (&red)[NW][NP], double* row) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        double v = gacc[q];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][q] = v;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NP; q += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < nwarps; ++w) v += red[w][q];
        row[q] = v;
    }
    __syncthreads();
}

template <class R, int METHOD, bool PP, int M>
__global__ void __launch_bounds__(256) adjoint_kernel(const __grid_constant__ AdjointArgs a) {
    constexpr int NP = R::NP;
    __shared__ double red[8][NP > 16 ? 1 : NP];  // per-warp partials (blocks of at most 256 threads)
    extern __shared__ float sts[];               // sweep_smem: M * D floats per thread
    double gacc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) gacc[q] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        adjoint_particle<R, METHOD, PP, M>(a, i, gacc, sts + threadIdx.x, blockDim.x);
    // per-block partial sums of the parameter gradient, in a fixed order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if constexpr (NP <= 16) {
        block_sum_to_row<NP, 8>(gacc, red, a.partial + (int64_t)blockIdx.x * a.np_stride);
    } else {
        // many parameters (the linear test system): one partial per warp, summed by the host-side pass
        for (int q = 0; q < NP; ++q) {
            double v = gacc[q];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) a.partial[((int64_t)blockIdx.x * nwarps + warp) * a.np_stride + q] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// Packed-pair adjoint for Lorenz RK4: two particles per thread in f32x2
// registers (lane 0 particle 2t, lane 1 particle 2t + 1).  Every operation is
// the scalar adjoint's, lane by lane (the shifted step, stage points, Jacobian
// products and reverse combination above), so dL/dx0 is the same to the bit
// and the parameter sums differ only in their FP64 order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ f2 mul2a(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

// LorenzShiftC per lane (lane 0 and lane 1 may differ in r, with a per-particle
// parameter, and in h, across a group boundary).
struct LorenzPairS {
    f2 s, ns, nb, nbr, nr, h1, h2, h6, nh1, nh2, nh6, sh1, sh2, sh6;
};

__device__ __forceinline__ LorenzPairS lorenz_pair(const LorenzShiftC& a, const LorenzShiftC& b) {
    LorenzPairS c;
    c.s = pack2(a.s, b.s);
    c.ns = pack2(a.ns, b.ns);
    c.nb = pack2(a.nb, b.nb);
    c.nbr = pack2(a.nbr, b.nbr);
    c.nr = pack2(a.nr, b.nr);
    c.h1 = pack2(a.h1, b.h1);
    c.h2 = pack2(a.h2, b.h2);
    c.h6 = pack2(a.h6, b.h6);
    c.nh1 = pack2(a.nh1, b.nh1);
    c.nh2 = pack2(a.nh2, b.nh2);
    c.nh6 = pack2(a.nh6, b.nh6);
    c.sh1 = pack2(a.sh1, b.sh1);
    c.sh2 = pack2(a.sh2, b.sh2);
    c.sh6 = pack2(a.sh6, b.sh6);
    return c;
}

// lorenz_shift_fwd lane by lane
__device__ __forceinline__ void lorenz_fwd2(f2 (&x)[3], const LorenzPairS& c) {
    const f2 two = pack2(2.0f, 2.0f);
    f2 d, A, kz, X, Y, Z, a0, a1, a2;
    d = sub2(x[1], x[0]);
    A = fma2(x[0], x[2], x[1]);
    kz = fma2(x[0], x[1], fma2(c.nb, x[2], c.nbr));
    a0 = d; a1 = A; a2 = kz;
    X = fma2(c.sh2, d, x[0]); Y = fma2(c.nh2, A, x[1]); Z = fma2(c.h2, kz, x[2]);
    d = sub2(Y, X);
    A = fma2(X, Z, Y);
    kz = fma2(X, Y, fma2(c.nb, Z, c.nbr));
    a0 = fma2(two, d, a0); a1 = fma2(two, A, a1); a2 = fma2(two, kz, a2);
    X = fma2(c.sh2, d, x[0]); Y = fma2(c.nh2, A, x[1]); Z = fma2(c.h2, kz, x[2]);
    d = sub2(Y, X);
    A = fma2(X, Z, Y);
    kz = fma2(X, Y, fma2(c.nb, Z, c.nbr));
    a0 = fma2(two, d, a0); a1 = fma2(two, A, a1); a2 = fma2(two, kz, a2);
    X = fma2(c.sh1, d, x[0]); Y = fma2(c.nh1, A, x[1]); Z = fma2(c.h1, kz, x[2]);
    d = sub2(Y, X);
    A = fma2(X, Z, Y);
    kz = fma2(X, Y, fma2(c.nb, Z, c.nbr));
    a0 = add2(a0, d); a1 = add2(a1, A); a2 = add2(a2, kz);
    x[0] = fma2(c.sh6, a0, x[0]); x[1] = fma2(c.nh6, a1, x[1]); x[2] = fma2(c.h6, a2, x[2]);
}

// lorenz_shift_stage lane by lane
__device__ __forceinline__ void lorenz_stage2(const f2 (&P)[3], const f2 (&x)[3], f2 cs, f2 cn, f2 ch,
                                              const LorenzPairS& c, f2 (&out)[3], f2& d) {
    d = sub2(P[1], P[0]);
    const f2 A = fma2(P[0], P[2], P[1]);
    const f2 kz = fma2(P[0], P[1], fma2(c.nb, P[2], c.nbr));
    out[0] = fma2(cs, d, x[0]);
    out[1] = fma2(cn, A, x[1]);
    out[2] = fma2(ch, kz, x[2]);
}

// lorenz_shift_vjp lane by lane (0 - v1 is the scalar's negation, also for a zero)
__device__ __forceinline__ void lorenz_vjp2(const f2 (&P)[3], f2 d, const LorenzPairS& c, const f2 (&v)[3],
                                            f2 (&jx)[3], f2 (&jp)[3]) {
    const f2 nv1 = sub2(pack2(0.0f, 0.0f), v[1]);
    jx[0] = fma2(c.ns, v[0], fma2(P[2], nv1, mul2a(P[1], v[2])));
    jx[1] = fma2(c.s, v[0], fma2(P[0], v[2], nv1));
    jx[2] = fma2(P[0], nv1, mul2a(c.nb, v[2]));
    jp[0] = fma2(d, v[0], jp[0]);
    jp[1] = fma2(P[0], v[1], jp[1]);
    jp[2] = fma2(sub2(c.nr, P[2]), v[2], jp[2]);
}

// lorenz_shift_adj lane by lane
__device__ __forceinline__ void lorenz_adj2(const f2 (&x)[3], f2 (&lam)[3], const LorenzPairS& c, f2 (&jp)[3]) {
    f2 x2[3], x3[3], x4[3], d1, d2, d3;
    lorenz_stage2(x, x, c.sh2, c.nh2, c.h2, c, x2, d1);
    lorenz_stage2(x2, x, c.sh2, c.nh2, c.h2, c, x3, d2);
    lorenz_stage2(x3, x, c.sh1, c.nh1, c.h1, c, x4, d3);
    const f2 d4 = sub2(x4[1], x4[0]);
    f2 u[3], u2[3], l[3], m[3], sum[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) { u[i] = mul2a(c.h6, lam[i]); u2[i] = add2(u[i], u[i]); }
    lorenz_vjp2(x4, d4, c, u, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = m[i]; l[i] = fma2(c.h1, m[i], u2[i]); }
    lorenz_vjp2(x3, d3, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = add2(sum[i], m[i]); l[i] = fma2(c.h2, m[i], u2[i]); }
    lorenz_vjp2(x2, d2, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = add2(sum[i], m[i]); l[i] = fma2(c.h2, m[i], u[i]); }
    lorenz_vjp2(x, d1, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[i] = add2(lam[i], add2(sum[i], m[i]));
}

// The states of the sub-segment being reversed live in shared memory, one
// 8-byte slot per thread and component ([step][component][thread], so a warp's
// accesses are consecutive), which keeps the register file for the arithmetic:
// 64-thread blocks, up to 8 resident per SM.
constexpr int kLx2Block = 64;

template <bool PP, int M>
__global__ void __launch_bounds__(kLx2Block, 8) adjoint_lorenz_x2_kernel(const __grid_constant__ AdjointArgs a) {
    __shared__ double red[kLx2Block / 32][3];
    __shared__ f2 st[M][3][kLx2Block];
    const int tid = threadIdx.x;
    double gacc[3] = {0.0, 0.0, 0.0};
    const int64_t npair = (a.n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npair; t += stride) {
        const int64_t i0 = 2 * t, i1 = 2 * t + 1;
        const bool has1 = i1 < a.n;  // an odd count leaves the last pair half empty
        int g0 = 0, g1 = 0;
#pragma unroll
        for (int q = 1; q < FF_MAX_GROUPS; ++q) {
            if (q < a.n_groups && i0 >= a.gstart[q]) g0 = q;
            if (q < a.n_groups && i1 >= a.gstart[q]) g1 = q;
        }
        f2 lam[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            lam[k] = pack2(a.lam_in[k * a.n + i0], has1 ? a.lam_in[k * a.n + i1] : 0.0f);
        const float pv0 = PP ? a.pparam[i0] : 0.0f, pv1 = (PP && has1) ? a.pparam[i1] : 0.0f;
        for (int c = a.n_chunks - 1; c >= 0; --c) {
            const AdjChunk& ch = a.chunks[c];
            float pa[3], pb[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                pa[q] = (PP && q == a.pidx) ? pv0 : ch.p[q];
                pb[q] = (PP && q == a.pidx) ? pv1 : ch.p[q];
            }
            LorenzShiftC ca, cb;
            ca.init(ch.gh[g0], pa);
            cb.init(ch.gh[g1], pb);
            const LorenzPairS cp2 = lorenz_pair(ca, cb);
            const int L = ch.n_steps;
            const float* ck = a.ckpt + (int64_t)ch.ckpt * a.dim * a.pitch;
            f2 x[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) x[k] = pack2(ck[k * a.pitch + i0], ck[k * a.pitch + i1]);  // pitch covers i1
            x[2] = sub2(x[2], pack2(pa[1], pb[1]));  // zt = z - r
            f2 cpt[M][3];
            int nsub = 0;
            for (int base = 0; base < L; base += M, ++nsub) {
#pragma unroll
                for (int k = 0; k < 3; ++k) cpt[nsub][k] = x[k];
                const int nq = (base + M < L) ? M : 0;
#pragma unroll 1
                for (int r = 0; r < nq; ++r) lorenz_fwd2(x, cp2);
            }
            f2 jp[3] = {pack2(0.f, 0.f), pack2(0.f, 0.f), pack2(0.f, 0.f)};
            for (int sq = nsub - 1; sq >= 0; --sq) {
                const int nq = min(M, L - sq * M);
#pragma unroll
                for (int k = 0; k < 3; ++k) x[k] = cpt[sq][k];
#pragma unroll
                for (int r = 0; r < M; ++r) {
                    if (r < nq) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) st[r][k][tid] = x[k];
                        if (r + 1 < nq) lorenz_fwd2(x, cp2);
                    }
                }
#pragma unroll
                for (int r = M - 1; r >= 0; --r)
                    if (r < nq) {
                        f2 xr[3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) xr[k] = st[r][k][tid];
                        lorenz_adj2(xr, lam, cp2, jp);
                    }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float u, w;
                unpack2(jp[q], u, w);
                gacc[q] += (double)u;
                if (has1) gacc[q] += (double)w;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float u, w;
            unpack2(lam[k], u, w);
            a.lam_out[k * a.n + i0] = u;
            if (has1) a.lam_out[k * a.n + i1] = w;
        }
    }
    block_sum_to_row<3, kLx2Block / 32>(gacc, red, a.partial + (int64_t)blockIdx.x * a.np_stride);
}

// ---------------------------------------------------------------------------
// Packed-pair sweep for chunks longer than 16 steps: sub-segments of 4 steps
// whose recomputation also keeps each step's three stage points, so the reverse
// step applies the four Jacobian products without recomputing them.  Per
// 64-thread block the 4 steps x (state + 3 stage points) take the 24.6 KB the
// 16 states of the plain sweep took; the sub-checkpoints (up to 64 per chunk)
// live in local memory.  The stage points are the ones lorenz_adj2 recomputes,
// operation for operation, so dL/dx0 is unchanged to the bit.
// ---------------------------------------------------------------------------
constexpr int kLx2sSub = 4;      // steps per sub-segment
constexpr int kLx2sMaxSub = 64;  // sub-checkpoints of a chunk of up to 256 steps

// lorenz_fwd2 that also returns the stage points x2, x3, x4 (S[3 s + k], component k of
// stage point s + 2); with full false the step's update is skipped.
__device__ __forceinline__ void lorenz_fwd2_stages(f2 (&x)[3], const LorenzPairS& c, f2 (&S)[9], bool full) {
    const f2 two = pack2(2.0f, 2.0f);
    f2 d, A, kz, X, Y, Z, a0, a1, a2;
    d = sub2(x[1], x[0]);
    A = fma2(x[0], x[2], x[1]);
    kz = fma2(x[0], x[1], fma2(c.nb, x[2], c.nbr));
    a0 = d; a1 = A; a2 = kz;
    X = fma2(c.sh2, d, x[0]); Y = fma2(c.nh2, A, x[1]); Z = fma2(c.h2, kz, x[2]);
    S[0] = X; S[1] = Y; S[2] = Z;
    d = sub2(Y, X);
    A = fma2(X, Z, Y);
    kz = fma2(X, Y, fma2(c.nb, Z, c.nbr));
    a0 = fma2(two, d, a0); a1 = fma2(two, A, a1); a2 = fma2(two, kz, a2);
    X = fma2(c.sh2, d, x[0]); Y = fma2(c.nh2, A, x[1]); Z = fma2(c.h2, kz, x[2]);
    S[3] = X; S[4] = Y; S[5] = Z;
    d = sub2(Y, X);
    A = fma2(X, Z, Y);
    kz = fma2(X, Y, fma2(c.nb, Z, c.nbr));
    a0 = fma2(two, d, a0); a1 = fma2(two, A, a1); a2 = fma2(two, kz, a2);
    X = fma2(c.sh1, d, x[0]); Y = fma2(c.nh1, A, x[1]); Z = fma2(c.h1, kz, x[2]);
    S[6] = X; S[7] = Y; S[8] = Z;
    if (!full) return;
    d = sub2(Y, X);
    A = fma2(X, Z, Y);
    kz = fma2(X, Y, fma2(c.nb, Z, c.nbr));
    a0 = add2(a0, d); a1 = add2(a1, A); a2 = add2(a2, kz);
    x[0] = fma2(c.sh6, a0, x[0]); x[1] = fma2(c.nh6, a1, x[1]); x[2] = fma2(c.h6, a2, x[2]);
}

// lorenz_adj2 with the stage points given (the same products and sums).
__device__ __forceinline__ void lorenz_adj2_given(const f2 (&x)[3], const f2 (&x2)[3], const f2 (&x3)[3],
                                                  const f2 (&x4)[3], f2 (&lam)[3], const LorenzPairS& c,
                                                  f2 (&jp)[3]) {
    const f2 d1 = sub2(x[1], x[0]), d2 = sub2(x2[1], x2[0]), d3 = sub2(x3[1], x3[0]), d4 = sub2(x4[1], x4[0]);
    f2 u[3], u2[3], l[3], m[3], sum[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) { u[i] = mul2a(c.h6, lam[i]); u2[i] = add2(u[i], u[i]); }
    lorenz_vjp2(x4, d4, c, u, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = m[i]; l[i] = fma2(c.h1, m[i], u2[i]); }
    lorenz_vjp2(x3, d3, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = add2(sum[i], m[i]); l[i] = fma2(c.h2, m[i], u2[i]); }
    lorenz_vjp2(x2, d2, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = add2(sum[i], m[i]); l[i] = fma2(c.h2, m[i], u[i]); }
    lorenz_vjp2(x, d1, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[i] = add2(lam[i], add2(sum[i], m[i]));
}

template <bool PP>
__global__ void __launch_bounds__(kLx2Block, 8) adjoint_lorenz_x2s_kernel(const __grid_constant__ AdjointArgs a) {
    constexpr int MS = kLx2sSub;
    __shared__ double red[kLx2Block / 32][3];
    __shared__ f2 st[MS][12][kLx2Block];  // per step: the state, then stage points 2, 3, 4
    const int tid = threadIdx.x;
    double gacc[3] = {0.0, 0.0, 0.0};
    const int64_t npair = (a.n + 1) / 2;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npair; t += stride) {
        const int64_t i0 = 2 * t, i1 = 2 * t + 1;
        const bool has1 = i1 < a.n;  // an odd count leaves the last pair half empty
        int g0 = 0, g1 = 0;
#pragma unroll
        for (int q = 1; q < FF_MAX_GROUPS; ++q) {
            if (q < a.n_groups && i0 >= a.gstart[q]) g0 = q;
            if (q < a.n_groups && i1 >= a.gstart[q]) g1 = q;
        }
        f2 lam[3];
#pragma unroll
        for (int k = 0; k < 3; ++k)
            lam[k] = pack2(a.lam_in[k * a.n + i0], has1 ? a.lam_in[k * a.n + i1] : 0.0f);
        const float pv0 = PP ? a.pparam[i0] : 0.0f, pv1 = (PP && has1) ? a.pparam[i1] : 0.0f;
        for (int c = a.n_chunks - 1; c >= 0; --c) {
            const AdjChunk& ch = a.chunks[c];
            float pa[3], pb[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                pa[q] = (PP && q == a.pidx) ? pv0 : ch.p[q];
                pb[q] = (PP && q == a.pidx) ? pv1 : ch.p[q];
            }
            LorenzShiftC ca, cb;
            ca.init(ch.gh[g0], pa);
            cb.init(ch.gh[g1], pb);
            const LorenzPairS cp2 = lorenz_pair(ca, cb);
            const int L = ch.n_steps;
            const float* ck = a.ckpt + (int64_t)ch.ckpt * a.dim * a.pitch;
            f2 x[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) x[k] = pack2(ck[k * a.pitch + i0], ck[k * a.pitch + i1]);  // pitch covers i1
            x[2] = sub2(x[2], pack2(pa[1], pb[1]));  // zt = z - r
            f2 cpt[kLx2sMaxSub][3];
            int nsub = 0;
            for (int base = 0; base < L; base += MS, ++nsub) {
#pragma unroll
                for (int k = 0; k < 3; ++k) cpt[nsub][k] = x[k];
                if (base + MS < L) {
#pragma unroll
                    for (int r = 0; r < MS; ++r) lorenz_fwd2(x, cp2);
                }
            }
            f2 jp[3] = {pack2(0.f, 0.f), pack2(0.f, 0.f), pack2(0.f, 0.f)};
            for (int sq = nsub - 1; sq >= 0; --sq) {
                const int nq = min(MS, L - sq * MS);
#pragma unroll
                for (int k = 0; k < 3; ++k) x[k] = cpt[sq][k];
#pragma unroll
                for (int r = 0; r < MS; ++r) {
                    if (r < nq) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) st[r][k][tid] = x[k];
                        f2 S[9];
                        lorenz_fwd2_stages(x, cp2, S, r + 1 < nq);
#pragma unroll
                        for (int k = 0; k < 9; ++k) st[r][3 + k][tid] = S[k];
                    }
                }
#pragma unroll
                for (int r = MS - 1; r >= 0; --r)
                    if (r < nq) {
                        f2 xr[3], x2[3], x3[3], x4[3];
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            xr[k] = st[r][k][tid];
                            x2[k] = st[r][3 + k][tid];
                            x3[k] = st[r][6 + k][tid];
                            x4[k] = st[r][9 + k][tid];
                        }
                        lorenz_adj2_given(xr, x2, x3, x4, lam, cp2, jp);
                    }
            }
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float u, w;
                unpack2(jp[q], u, w);
                gacc[q] += (double)u;
                if (has1) gacc[q] += (double)w;
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float u, w;
            unpack2(lam[k], u, w);
            a.lam_out[k * a.n + i0] = u;
            if (has1) a.lam_out[k * a.n + i1] = w;
        }
    }
    block_sum_to_row<3, kLx2Block / 32>(gacc, red, a.partial + (int64_t)blockIdx.x * a.np_stride);
}

// Batched adjoint: each block takes tiles round-robin; a tile is a run of
// particles of one member, one per thread, and its parameter gradient is
// reduced over the block into the tile's own row.
template <class R, int METHOD, bool PP, int M>
__global__ void __launch_bounds__(kAdjTile) batch_adjoint_kernel(const __grid_constant__ BatchAdjointArgs b) {
    constexpr int NP = R::NP;
    __shared__ double red[kAdjTile / 32][NP];
    extern __shared__ float sts[];  // sweep_smem: M * D floats per thread
    for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
        const AdjTile T = b.tiles[tile];
        const AdjointArgs& a = b.sys[T.sys];
        double gacc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) gacc[q] = 0.0;
        const int64_t i = T.first + threadIdx.x;
        if (i < T.first + T.count) adjoint_particle<R, METHOD, PP, M>(a, i, gacc, sts + threadIdx.x, kAdjTile);
        block_sum_to_row<NP, kAdjTile / 32>(gacc, red, b.partial + (int64_t)tile * b.np_stride);
    }
}

template <class R, int METHOD, bool PP, int M>
static cudaError_t launch_batch_one(const BatchAdjointArgs& b, int num_sms, cudaStream_t s) {
    auto kernel = batch_adjoint_kernel<R, METHOD, PP, M>;
    const size_t smem = sweep_smem<R, M>(kAdjTile);
    cudaError_t e = allow_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kAdjTile, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t cap = (int64_t)occ * num_sms;
    const int grid = (int)((int64_t)b.n_tiles < cap ? b.n_tiles : cap);
    if (grid < 1) return cudaSuccess;
    kernel<<<grid, kAdjTile, smem, s>>>(b);
    return cudaGetLastError();
}

template <class R, int M>
static cudaError_t launch_batch_m(int method, bool pp, const BatchAdjointArgs& b, int num_sms, cudaStream_t s) {
    if (method == FF_RK4)
        return pp ? launch_batch_one<R, FF_RK4, true, M>(b, num_sms, s) : launch_batch_one<R, FF_RK4, false, M>(b, num_sms, s);
    return pp ? launch_batch_one<R, FF_EULER, true, M>(b, num_sms, s) : launch_batch_one<R, FF_EULER, false, M>(b, num_sms, s);
}

template <class R>
static cudaError_t launch_batch_r(int method, bool pp, int m, const BatchAdjointArgs& b, int num_sms, cudaStream_t s) {
    switch (m) {
    case 4: return launch_batch_m<R, 4>(method, pp, b, num_sms, s);
    case 8: return launch_batch_m<R, 8>(method, pp, b, num_sms, s);
    case 16: return launch_batch_m<R, 16>(method, pp, b, num_sms, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class R, int METHOD, bool PP, int M>
static cudaError_t launch_one(const AdjointArgs& a0, int block, int num_sms, cudaStream_t s, int64_t* rows) {
    AdjointArgs a = a0;
    auto kernel = adjoint_kernel<R, METHOD, PP, M>;
    const size_t smem = sweep_smem<R, M>(block);
    cudaError_t e = allow_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t need = (a.n + block - 1) / block;
    int64_t cap = (int64_t)occ * num_sms;
    if (cap > a.max_blocks) cap = a.max_blocks;  // rows of the partial-sum buffer
    const int grid = (int)(need < cap ? need : cap);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    kernel<<<grid, block, smem, s>>>(a);
    *rows = R::NP <= 16 ? grid : (int64_t)grid * (block / 32);
    return cudaGetLastError();
}

template <class R, int M>
static cudaError_t launch_m(int method, bool pp, const AdjointArgs& a, int block, int num_sms, cudaStream_t s,
                            int64_t* rows) {
    if (method == FF_RK4)
        return pp ? launch_one<R, FF_RK4, true, M>(a, block, num_sms, s, rows)
                  : launch_one<R, FF_RK4, false, M>(a, block, num_sms, s, rows);
    return pp ? launch_one<R, FF_EULER, true, M>(a, block, num_sms, s, rows)
              : launch_one<R, FF_EULER, false, M>(a, block, num_sms, s, rows);
}

template <class R>
static cudaError_t launch_r(int method, bool pp, int m, const AdjointArgs& a, int block, int num_sms, cudaStream_t s,
                            int64_t* rows) {
    switch (m) {
    case 4: return launch_m<R, 4>(method, pp, a, block, num_sms, s, rows);
    case 8: return launch_m<R, 8>(method, pp, a, block, num_sms, s, rows);
    case 16: return launch_m<R, 16>(method, pp, a, block, num_sms, s, rows);
    default: return cudaErrorInvalidValue;
    }
}

template <class Kernel>
static cudaError_t launch_lorenz_x2_kernel(Kernel kernel, const AdjointArgs& a, int num_sms, cudaStream_t s,
                                           int64_t* rows) {
    // the sub-segment states take shared memory, so favour it over L1
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kLx2Block, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t need = ((a.n + 1) / 2 + kLx2Block - 1) / kLx2Block;
    int64_t cap = (int64_t)occ * num_sms;
    if (cap > 8 * a.max_blocks) cap = 8 * a.max_blocks;  // rows of the partial-sum buffer (one per block here)
    const int grid = (int)(need < cap ? need : cap);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    kernel<<<grid, kLx2Block, 0, s>>>(a);
    *rows = grid;
    return cudaGetLastError();
}

template <bool PP, int M>
static cudaError_t launch_lorenz_x2_one(const AdjointArgs& a, int num_sms, cudaStream_t s, int64_t* rows) {
    return launch_lorenz_x2_kernel(adjoint_lorenz_x2_kernel<PP, M>, a, num_sms, s, rows);
}

}  // namespace ff
