// ff_adjoint_impl.cuh -- device code and launch templates of the discrete
// adjoint of the RK4 / Euler integrator (not part of the paper), shared by the
// per-family translation units (ff_adjoint_lorenz.cu, ff_adjoint_hh3.cu,
// ff_adjoint_small.cu, ff_adjoint_linear.cu), which compile in parallel.
//
// One thread per particle walks the chunks in reverse with the adjoint state
// lambda = dL/dx in registers.  A chunk of L <= M*M steps is recomputed from its
// checkpoint twice (once when L <= M): once to place sub-checkpoints every M
// steps (local memory), then per sub-segment (in reverse) to put its <= M
// states in registers (shared memory in the packed Lorenz sweep), which the
// reverse RK4 steps consume from last to first.  The 15-dimensional system runs
// the staged sweep instead: one recomputation per chunk into a global scratch.  Parameter gradients are summed
// per particle in FP32 within a chunk, added to FP64 per chunk, and reduced
// over particles through per-block FP64 partials in fixed order.
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

// Parameter-derived constants of the HH3 vector-Jacobian product, per lane type.
template <class O> struct HHVjpConst {
    typename O::T gNa, gK, gL, ENa, EK, EL, gsyn, Esyn, invC, neg_invC, inv_tr, neg_inv_tr, neg_inv_td,
        inv_td2, sig, neg_sig, neg_sig2, sig2_theta, theta, gNa3, gK4;
};

template <class O>
__device__ __forceinline__ HHVjpConst<O> hh_vjp_const(const float* p) {
    HHVjpConst<O> c;
    const float invC = __fdividef(1.0f, p[0]), inv_tr = __fdividef(1.0f, p[12]), inv_td = __fdividef(1.0f, p[13]);
    const float sig2 = p[14] * kLog2e;
    c.gNa = O::k(p[1]);
    c.gK = O::k(p[2]);
    c.gL = O::k(p[3]);
    c.ENa = O::k(p[4]);
    c.EK = O::k(p[5]);
    c.EL = O::k(p[6]);
    c.gsyn = O::k(p[7]);
    c.Esyn = O::k(p[8]);
    c.invC = O::k(invC);
    c.neg_invC = O::k(-invC);
    c.inv_tr = O::k(inv_tr);
    c.neg_inv_tr = O::k(-inv_tr);
    c.neg_inv_td = O::k(-inv_td);
    c.inv_td2 = O::k(inv_td * inv_td);
    c.sig = O::k(p[14]);
    c.neg_sig = O::k(-p[14]);
    c.neg_sig2 = O::k(-sig2);
    c.sig2_theta = O::k(sig2 * p[15]);
    c.theta = O::k(p[15]);
    c.gNa3 = O::k(3.0f * p[1]);
    c.gK4 = O::k(4.0f * p[2]);
    return c;
}

// d/dy of y / (1 - e^-y) by its series 1/2 + y/6 - y^3/180 + y^5/5040 - y^7/151200 (|y| < 0.5).
template <class O>
__device__ __forceinline__ typename O::T bernoulli_series_deriv_t(typename O::T y) {
    const auto y2 = O::mul(y, y);
    return O::fma(y, O::fma(y2, O::fma(y2, O::fma(y2, O::k(-1.0f / 151200.0f), O::k(1.0f / 5040.0f)),
                                       O::k(-1.0f / 180.0f)), O::k(1.0f / 6.0f)), O::k(0.5f));
}

// One neuron of the HH3 vector-Jacobian product (Eq. 6-11 differentiated term by
// term; the gate rates depend on V only), over a lane type.  With u = v_V / C:
//   jx_V = sum over gates of v_y (a'(1 - y) - b' y) + v_s sig act (1 - act)(1 - s) / tau_r
//          - u (gL + gNa m^3 h + gK n^4 + gsyn S)
//   jx_y = (the current term's derivative) u - v_y (a + b)       for y = m, h, n
//   self = -v_s (act / tau_r + 1 / tau_d)   (the own-s part of jx_s)
//   syn  = gsyn (Esyn - V) u                 (added to the other neurons' jx_s)
// and the neuron's contributions cp to dL/dp (indices 0..8, its drive, 12..15).
template <class O>
__device__ __forceinline__ void hh_neuron_vjp(typename O::T V, typename O::T m, typename O::T h, typename O::T n,
                                              typename O::T s, typename O::T others, typename O::T drive,
                                              typename O::T uV, typename O::T vm, typename O::T vh,
                                              typename O::T vn, typename O::T vs, const HHVjpConst<O>& c,
                                              typename O::T (&jx)[4], typename O::T& self, typename O::T& syn,
                                              typename O::T (&cp)[14]) {
    using T = typename O::T;
    constexpr float kE25 = 12.182493960703473f;  // e^2.5
    constexpr float kE1 = 2.718281828459045f;    // e^1
    constexpr float kE3 = 20.085536923187668f;   // e^3
    constexpr float kQ = -kLog2e / 80.0f, kQ0 = 65.0f * (-kLog2e / 80.0f);
    constexpr float kB = -kLog2e / 18.0f, kB0 = 65.0f * (-kLog2e / 18.0f) + 2.0f;
    const T one = O::k(1.0f);
    // rates and their derivatives (the rates as in the forward right-hand side)
    const T q = O::ex2(O::fma(V, O::k(kQ), O::k(kQ0)));
    const T q2 = O::mul(q, q), q4 = O::mul(q2, q2), q8 = O::mul(q4, q4);
    const T bm = O::ex2(O::fma(V, O::k(kB), O::k(kB0)));
    const T ah = O::mul(O::k(0.07f), q4);
    const T bn = O::mul(O::k(0.125f), q);
    const T es = O::ex2(O::fma(c.neg_sig2, V, c.sig2_theta));
    const T ym = O::fma(V, O::k(0.1f), O::k(4.0f)), yn = O::fma(V, O::k(0.1f), O::k(5.5f));
    const auto sm = O::small(ym), sn = O::small(yn);
    const T em = O::mul(O::k(kE25), q8), en = O::mul(O::k(kE1), q8);
    const T dm = O::sel(sm, one, O::sub(one, em)), dn = O::sel(sn, one, O::sub(one, en));
    const T rmn = O::rcp(O::mul(dm, dn));
    const T rm = O::mul(dn, rmn), rn = O::mul(dm, rmn);  // 1 / dm, 1 / dn
    // g(y) = y / (1 - e^-y), g'(y) = (1 - e^-y (1 + y)) / (1 - e^-y)^2; alpha_m = g(ym), alpha_n = g(yn) / 10
    // at most one of ym, yn (which differ by 1.5) lies in the series band: one series and one
    // derivative series serve both
    const T ys = O::sel(sm, ym, yn);
    const T ser = bernoulli_series_t<O>(ys), dser = bernoulli_series_deriv_t<O>(ys);
    const T am = O::sel(sm, ser, O::mul(ym, rm));
    const T gn = O::sel(sn, ser, O::mul(yn, rn));
    const T dgm = O::sel(sm, dser, O::mul(O::fms(em, O::add(one, ym), one), O::mul(rm, rm)));
    const T dgn = O::sel(sn, dser, O::mul(O::fms(en, O::add(one, yn), one), O::mul(rn, rn)));
    const T anbn = O::fma(O::k(0.1f), gn, bn);  // alpha_n + beta_n (alpha_n = g(yn) / 10), fused
    const T dam = O::mul(O::k(0.1f), dgm), dan = O::mul(O::k(0.01f), dgn);
    const T ph = O::fma(O::k(kE3), q8, one), ps = O::add(one, es);
    const T r = O::rcp(O::mul(ph, ps));
    const T bh = O::mul(ps, r), act = O::mul(ph, r);
    const T a1 = O::mul(act, O::sub(one, act));
    // minus the beta derivatives: beta_m' = -beta_m/18, beta_n' = -beta_n/80, beta_h' = beta_h (1 - beta_h)/10
    const T nd_bm = O::mul(bm, O::k(1.0f / 18.0f)), nd_bn = O::mul(bn, O::k(1.0f / 80.0f));
    const T nd_bh = O::mul(O::mul(O::k(0.1f), bh), O::sub(bh, one));
    const T dah = O::mul(ah, O::k(-1.0f / 20.0f));
    // currents
    const T m2 = O::mul(m, m), m3 = O::mul(m2, m), m3h = O::mul(m3, h);
    const T n2 = O::mul(n, n), n3 = O::mul(n2, n), n4 = O::mul(n2, n2);
    const T dNa = O::sub(c.ENa, V), dK = O::sub(c.EK, V), dL = O::sub(c.EL, V), dS = O::sub(c.Esyn, V);
    T I = O::mul(c.gL, dL);
    I = O::fma(O::mul(c.gNa, m3h), dNa, I);
    I = O::fma(O::mul(c.gK, n4), dK, I);
    I = O::fma(O::mul(c.gsyn, others), dS, I);
    I = O::add(I, drive);
    const T gtot = O::fma(c.gsyn, others, O::fma(c.gK, n4, O::fma(c.gNa, m3h, c.gL)));
    // state
    const T sv = O::mul(O::mul(vs, c.inv_tr), O::sub(one, s));  // v_s (1 - s) / tau_r
    const T gate_m = O::fma(dam, O::sub(one, m), O::mul(nd_bm, m));
    const T gate_h = O::fma(dah, O::sub(one, h), O::mul(nd_bh, h));
    const T gate_n = O::fma(dan, O::sub(one, n), O::mul(nd_bn, n));
    const T jv = O::fma(vm, gate_m, O::fma(vh, gate_h, O::fma(vn, gate_n, O::mul(O::mul(c.sig, a1), sv))));
    // x - u w with one rounding (O::fms)
    jx[0] = O::fms(uV, gtot, jv);
    jx[1] = O::fms(vm, O::add(am, bm), O::mul(O::mul(O::mul(O::mul(uV, c.gNa3), m2), h), dNa));
    jx[2] = O::fms(vh, O::add(ah, bh), O::mul(O::mul(O::mul(uV, c.gNa), m3), dNa));
    jx[3] = O::fms(vn, anbn, O::mul(O::mul(O::mul(uV, c.gK4), n3), dK));
    self = O::mul(vs, O::fma(act, c.neg_inv_tr, c.neg_inv_td));
    syn = O::mul(O::mul(c.gsyn, dS), uV);
    // parameters: C, gNa, gK, gL, ENa, EK, EL, gsyn, Esyn, drive, tau_r, tau_d, sig, theta
    cp[0] = O::mul(O::mul(I, c.neg_invC), uV);
    cp[1] = O::mul(O::mul(m3h, dNa), uV);
    cp[2] = O::mul(O::mul(n4, dK), uV);
    cp[3] = O::mul(dL, uV);
    cp[4] = O::mul(O::mul(c.gNa, m3h), uV);
    cp[5] = O::mul(O::mul(c.gK, n4), uV);
    cp[6] = O::mul(c.gL, uV);
    cp[7] = O::mul(O::mul(dS, others), uV);
    cp[8] = O::mul(O::mul(c.gsyn, others), uV);
    cp[9] = uV;
    cp[10] = O::mul(O::mul(act, c.neg_inv_tr), sv);
    cp[11] = O::mul(O::mul(s, c.inv_td2), vs);
    cp[12] = O::mul(O::mul(a1, O::sub(V, c.theta)), sv);
    cp[13] = O::mul(O::mul(c.neg_sig, a1), sv);
}

template <> struct Vjp<HH3> {
    // Neurons 0 and 1 run the neuron product above packed in f32x2 registers,
    // neuron 2 on floats, with the same operations.  The gate rows of jx can still
    // round one way in f32x2 and another in floats (measured: about a quarter of
    // random inputs, by one rounding), where the toolchain fuses a different pair
    // of packed operations than the float form; every kernel runs this same code,
    // so batched and standalone sweeps agree to the bit.
    __device__ __forceinline__ static void apply(const float (&x)[15], const float* p, const float (&v)[15],
                                                 float (&jx)[15], float* jp) {
        const HHVjpConst<HHPair> c2 = hh_vjp_const<HHPair>(p);
        const HHVjpConst<HHScalar> c1 = hh_vjp_const<HHScalar>(p);
        const float s_sum = __fadd_rn(__fadd_rn(x[4], x[9]), x[14]);
        const f2 S01 = pack2(x[4], x[9]);
        const f2 uV01 = mul2(pack2(v[0], v[5]), c2.invC);
        f2 jx01[4], self01, syn01, cp01[14];
        hh_neuron_vjp<HHPair>(pack2(x[0], x[5]), pack2(x[1], x[6]), pack2(x[2], x[7]), pack2(x[3], x[8]), S01,
                              sub2(pack2(s_sum, s_sum), S01), pack2(p[9], p[10]), uV01, pack2(v[1], v[6]),
                              pack2(v[2], v[7]), pack2(v[3], v[8]), pack2(v[4], v[9]), c2, jx01, self01, syn01, cp01);
        float jx2[4], self2, syn2, cp2[14];
        hh_neuron_vjp<HHScalar>(x[10], x[11], x[12], x[13], x[14], __fsub_rn(s_sum, x[14]), p[11],
                                __fmul_rn(v[10], c1.invC), v[11], v[12], v[13], v[14], c1, jx2, self2, syn2, cp2);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            unpack2(jx01[k], jx[k], jx[5 + k]);
            jx[10 + k] = jx2[k];
        }
        float self0, self1, syn0, syn1;
        unpack2(self01, self0, self1);
        unpack2(syn01, syn0, syn1);
        const float syn_sum = __fadd_rn(__fadd_rn(syn0, syn1), syn2);
        jx[4] = __fadd_rn(self0, __fsub_rn(syn_sum, syn0));
        jx[9] = __fadd_rn(self1, __fsub_rn(syn_sum, syn1));
        jx[14] = __fadd_rn(self2, __fsub_rn(syn_sum, syn2));
        // parameter contributions: neuron 0 + neuron 1 + neuron 2 (drives: one each)
        float a0[14], a1[14];
#pragma unroll
        for (int k = 0; k < 14; ++k) unpack2(cp01[k], a0[k], a1[k]);
#pragma unroll
        for (int k = 0; k < 9; ++k) jp[k] = __fadd_rn(jp[k], __fadd_rn(__fadd_rn(a0[k], a1[k]), cp2[k]));
        jp[9] = __fadd_rn(jp[9], a0[9]);
        jp[10] = __fadd_rn(jp[10], a1[9]);
        jp[11] = __fadd_rn(jp[11], cp2[9]);
#pragma unroll
        for (int k = 10; k < 14; ++k) jp[k + 2] = __fadd_rn(jp[k + 2], __fadd_rn(__fadd_rn(a0[k], a1[k]), cp2[k]));
    }
};

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
    }
    const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
    static_assert(METHOD == FF_EULER || D <= 8, "the 15-dimensional system's reverse RK4 step is adj_step_staged");
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

// Reverse sweep of one particle i over all chunks: lambda from lam_in to
// lam_out, parameter contributions added to gacc (FP64, per chunk).  For systems
// of up to 8 dimensions (the 15-dimensional one runs adjoint_particle_staged).
template <class R, int METHOD, bool PP, int M>
__device__ __forceinline__ void adjoint_particle(const AdjointArgs& a, int64_t i, double (&gacc)[R::NP]) {
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
            float st[M][D];
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = cp[sq][k];
#pragma unroll
            for (int r = 0; r < M; ++r) {
                if (r < nq) {
#pragma unroll
                    for (int k = 0; k < D; ++k) st[r][k] = x[k];
                    if (r + 1 < nq) fwd_step<R, METHOD>(x, h, p);
                }
            }
#pragma unroll
            for (int r = M - 1; r >= 0; --r)
                if (r < nq) adj_step<R, METHOD>(st[r], lam, h, p, jp);
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
    double gacc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) gacc[q] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride)
        adjoint_particle<R, METHOD, PP, M>(a, i, gacc);
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
// Staged sweep for the 15-dimensional system (HH x 3).  Its sub-segment states
// do not fit in registers, so a chunk is recomputed once from its checkpoint
// and every state goes to the thread's scratch area in global memory (state
// variable k of step r at scratch[(r * D + k) * T], T the launch's threads: one
// coalesced column per warp); the reverse steps read them back from last to
// first.  The reverse step's three stage points live in shared memory, and the
// kernels run 4 blocks of 128 threads per SM within the register file.  Against
// the two-level scheme of adjoint_particle this saves one forward
// recomputation per step; the states, steps and sums are the same, in the same
// order, so the gradients agree with it to the bit.
// ---------------------------------------------------------------------------
constexpr int kStagedBlock = 128;
constexpr int kStagedMinBlocks = 3;

// adj_step with the step's state and its RK4 stage points in shared memory:
// stage + (s * D + i) * bs holds component i of stage point s + 1 (x1 = x) for this
// thread, and the parameter contributions accumulate in jp + q * bs (shared).
template <class R, int METHOD>
__device__ __forceinline__ void adj_step_staged(float (&xs)[R::DIM], float (&lam)[R::DIM], float h, const float* p,
                                                float* jp, float* stage, int bs) {
    constexpr int D = R::DIM, NP = R::NP;
    float jr[NP];
    if constexpr (METHOD == FF_EULER) {
#pragma unroll
        for (int q = 0; q < NP; ++q) jr[q] = jp[q * bs];
        adj_step<R, METHOD>(xs, lam, h, p, jr);
#pragma unroll
        for (int q = 0; q < NP; ++q) jp[q * bs] = jr[q];
    } else {
        const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
        float k[D], l[D], m[D], sum[D];
#pragma unroll
        for (int i = 0; i < D; ++i) stage[i * bs] = xs[i];
#pragma unroll 1
        for (int st = 0; st < 3; ++st) {
            if constexpr (std::is_same<R, HH3>::value) hh3_f_packed(xs, p, k);  // the bits of HH3::f
            else R::f(xs, p, k);
            const float c = (st == 2) ? h : h2;
#pragma unroll
            for (int i = 0; i < D; ++i) {
                xs[i] = fmaf(c, k[i], stage[i * bs]);
                stage[((st + 1) * D + i) * bs] = xs[i];
            }
        }
#pragma unroll 1
        for (int st = 3; st >= 0; --st) {
            if (st == 3) {
#pragma unroll
                for (int i = 0; i < D; ++i) l[i] = h6 * lam[i];
            } else {
                const float cl = (st == 0) ? h6 : h3, cm = (st == 2) ? h : h2;
#pragma unroll
                for (int i = 0; i < D; ++i) l[i] = fmaf(cl, lam[i], cm * m[i]);
            }
#pragma unroll
            for (int i = 0; i < D; ++i) xs[i] = stage[(st * D + i) * bs];
#pragma unroll
            for (int q = 0; q < NP; ++q) jr[q] = jp[q * bs];
            Vjp<R>::apply(xs, p, l, m, jr);
#pragma unroll
            for (int q = 0; q < NP; ++q) jp[q * bs] = jr[q];
            if (st == 3) {
#pragma unroll
                for (int i = 0; i < D; ++i) sum[i] = m[i];
            } else if (st > 0) {
#pragma unroll
                for (int i = 0; i < D; ++i) sum[i] = __fadd_rn(sum[i], m[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < D; ++i) lam[i] = __fadd_rn(lam[i], __fadd_rn(sum[i], m[i]));
    }
}

// Reverse sweep of particle i with the chunk's states in the thread's scratch
// (scr = the thread's first float, T = floats between consecutive entries); stage
// and jp are the thread's shared-memory columns (stride bs).
template <class R, int METHOD, bool PP>
__device__ __forceinline__ void adjoint_particle_staged(const AdjointArgs& a, int64_t i, double (&gacc)[R::NP],
                                                        float* scr, int64_t T, float* stage, float* jp, int bs) {
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
        // the chunk's parameters: read from the chunk table where they are the same for every
        // particle (the compiler may load them again where needed instead of holding them)
        float pl[PP ? NP : 1];
        if constexpr (PP) {
#pragma unroll
            for (int q = 0; q < NP; ++q) pl[q] = (q == a.pidx) ? pv : ch.p[q];
        }
        const float* p = PP ? pl : ch.p;
        const float h = ch.gh[g];
        const int L = ch.n_steps;
        const float* ck = a.ckpt + (int64_t)ch.ckpt * a.dim * a.pitch;
        float x[D];
#pragma unroll
        for (int k = 0; k < D; ++k) x[k] = (k < a.dim) ? ck[k * a.pitch + i] : 0.0f;
#pragma unroll 1
        for (int r = 0; r < L; ++r) {
#pragma unroll
            for (int k = 0; k < D; ++k) scr[((int64_t)r * D + k) * T] = x[k];
            if (r + 1 < L) fwd_step<R, METHOD>(x, h, p);
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) jp[q * bs] = 0.0f;
#pragma unroll 1
        for (int r = L - 1; r >= 0; --r) {
#pragma unroll
            for (int k = 0; k < D; ++k) x[k] = scr[((int64_t)r * D + k) * T];
            adj_step_staged<R, METHOD>(x, lam, h, p, jp, stage, bs);
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) gacc[q] += (double)jp[q * bs];
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
        if (k < a.dim) a.lam_out[k * a.n + i] = lam[k];
}

template <class R, int METHOD, bool PP>
__global__ void __launch_bounds__(kStagedBlock, kStagedMinBlocks) adjoint_staged_kernel(
    const __grid_constant__ AdjointArgs a) {
    constexpr int NP = R::NP, D = R::DIM;
    __shared__ double red[kStagedBlock / 32][NP];
    __shared__ float stage[4 * D * kStagedBlock];
    __shared__ float jp[NP * kStagedBlock];
    double gacc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) gacc[q] = 0.0;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = t; i < a.n; i += T)
        adjoint_particle_staged<R, METHOD, PP>(a, i, gacc, a.scratch + t, T, stage + threadIdx.x, jp + threadIdx.x,
                                               blockDim.x);
    block_sum_to_row<NP, kStagedBlock / 32>(gacc, red, a.partial + (int64_t)blockIdx.x * a.np_stride);
}

// Batched form: tiles of one member's particles, one per thread, round-robin over the blocks.
template <class R, int METHOD, bool PP>
__global__ void __launch_bounds__(kAdjTile, kStagedMinBlocks) batch_adjoint_staged_kernel(
    const __grid_constant__ BatchAdjointArgs b) {
    constexpr int NP = R::NP, D = R::DIM;
    static_assert(kAdjTile == kStagedBlock, "one tile per block");
    __shared__ double red[kAdjTile / 32][NP];
    __shared__ float stage[4 * D * kAdjTile];
    __shared__ float jp[NP * kAdjTile];
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
        const AdjTile tl = b.tiles[tile];
        const AdjointArgs& a = b.sys[tl.sys];
        double gacc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) gacc[q] = 0.0;
        const int64_t i = tl.first + threadIdx.x;
        if (i < tl.first + tl.count)
            adjoint_particle_staged<R, METHOD, PP>(a, i, gacc, b.scratch + t, T, stage + threadIdx.x,
                                                   jp + threadIdx.x, blockDim.x);
        block_sum_to_row<NP, kAdjTile / 32>(gacc, red, b.partial + (int64_t)tile * b.np_stride);
    }
}

// Resident threads of a staged kernel: the most it launches, and the scratch it needs room for.
template <class Kernel>
static int64_t staged_threads(Kernel kernel, int num_sms) {
    int occ = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kStagedBlock, 0) != cudaSuccess || occ < 1)
        return 0;
    return (int64_t)occ * num_sms * kStagedBlock;
}

template <class R, bool BATCHED>
static int64_t staged_threads_for(int method, bool pp, int num_sms) {
    if constexpr (BATCHED) {
        if (method == FF_RK4)
            return pp ? staged_threads(batch_adjoint_staged_kernel<R, FF_RK4, true>, num_sms)
                      : staged_threads(batch_adjoint_staged_kernel<R, FF_RK4, false>, num_sms);
        return pp ? staged_threads(batch_adjoint_staged_kernel<R, FF_EULER, true>, num_sms)
                  : staged_threads(batch_adjoint_staged_kernel<R, FF_EULER, false>, num_sms);
    } else {
        if (method == FF_RK4)
            return pp ? staged_threads(adjoint_staged_kernel<R, FF_RK4, true>, num_sms)
                      : staged_threads(adjoint_staged_kernel<R, FF_RK4, false>, num_sms);
        return pp ? staged_threads(adjoint_staged_kernel<R, FF_EULER, true>, num_sms)
                  : staged_threads(adjoint_staged_kernel<R, FF_EULER, false>, num_sms);
    }
}

template <class R, int METHOD, bool PP>
static cudaError_t launch_staged_one(const AdjointArgs& a, int num_sms, cudaStream_t s, int64_t* rows) {
    auto kernel = adjoint_staged_kernel<R, METHOD, PP>;
    const int64_t resident = staged_threads(kernel, num_sms);
    if (resident < kStagedBlock) return cudaErrorInvalidConfiguration;
    int64_t cap = resident / kStagedBlock;
    if (cap > a.scratch_threads / kStagedBlock) cap = a.scratch_threads / kStagedBlock;  // room in the scratch
    if (cap > 8 * a.max_blocks) cap = 8 * a.max_blocks;  // rows of the partial-sum buffer (one per block here)
    const int64_t need = (a.n + kStagedBlock - 1) / kStagedBlock;
    const int grid = (int)(need < cap ? need : cap);
    if (grid < 1 || !a.scratch) return cudaErrorInvalidConfiguration;
    kernel<<<grid, kStagedBlock, 0, s>>>(a);
    *rows = grid;
    return cudaGetLastError();
}

template <class R>
static cudaError_t launch_staged(int method, bool pp, const AdjointArgs& a, int num_sms, cudaStream_t s,
                                 int64_t* rows) {
    if (method == FF_RK4)
        return pp ? launch_staged_one<R, FF_RK4, true>(a, num_sms, s, rows)
                  : launch_staged_one<R, FF_RK4, false>(a, num_sms, s, rows);
    return pp ? launch_staged_one<R, FF_EULER, true>(a, num_sms, s, rows)
              : launch_staged_one<R, FF_EULER, false>(a, num_sms, s, rows);
}

template <class R, int METHOD, bool PP>
static cudaError_t launch_batch_staged_one(const BatchAdjointArgs& b, int num_sms, cudaStream_t s) {
    auto kernel = batch_adjoint_staged_kernel<R, METHOD, PP>;
    const int64_t resident = staged_threads(kernel, num_sms);
    if (resident < kAdjTile) return cudaErrorInvalidConfiguration;
    int64_t cap = resident / kAdjTile;
    if (cap > b.scratch_threads / kAdjTile) cap = b.scratch_threads / kAdjTile;
    const int grid = (int)((int64_t)b.n_tiles < cap ? b.n_tiles : cap);
    if (grid < 1) return cudaSuccess;
    if (!b.scratch) return cudaErrorInvalidConfiguration;
    kernel<<<grid, kAdjTile, 0, s>>>(b);
    return cudaGetLastError();
}

template <class R>
static cudaError_t launch_batch_staged(int method, bool pp, const BatchAdjointArgs& b, int num_sms, cudaStream_t s) {
    if (method == FF_RK4)
        return pp ? launch_batch_staged_one<R, FF_RK4, true>(b, num_sms, s)
                  : launch_batch_staged_one<R, FF_RK4, false>(b, num_sms, s);
    return pp ? launch_batch_staged_one<R, FF_EULER, true>(b, num_sms, s)
              : launch_batch_staged_one<R, FF_EULER, false>(b, num_sms, s);
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
                const int nq = (base + MS < L) ? MS : 0;
#pragma unroll 1
                for (int r = 0; r < nq; ++r) lorenz_fwd2(x, cp2);
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
    for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
        const AdjTile T = b.tiles[tile];
        const AdjointArgs& a = b.sys[T.sys];
        double gacc[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) gacc[q] = 0.0;
        const int64_t i = T.first + threadIdx.x;
        if (i < T.first + T.count) adjoint_particle<R, METHOD, PP, M>(a, i, gacc);
        block_sum_to_row<NP, kAdjTile / 32>(gacc, red, b.partial + (int64_t)tile * b.np_stride);
    }
}

template <class R, int METHOD, bool PP, int M>
static cudaError_t launch_batch_one(const BatchAdjointArgs& b, int num_sms, cudaStream_t s) {
    auto kernel = batch_adjoint_kernel<R, METHOD, PP, M>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kAdjTile, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t cap = (int64_t)occ * num_sms;
    const int grid = (int)((int64_t)b.n_tiles < cap ? b.n_tiles : cap);
    if (grid < 1) return cudaSuccess;
    kernel<<<grid, kAdjTile, 0, s>>>(b);
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
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    int64_t need = (a.n + block - 1) / block;
    int64_t cap = (int64_t)occ * num_sms;
    if (cap > a.max_blocks) cap = a.max_blocks;  // rows of the partial-sum buffer
    const int grid = (int)(need < cap ? need : cap);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    kernel<<<grid, block, 0, s>>>(a);
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

static cudaError_t launch_lorenz_x2(bool pp, int m, const AdjointArgs& a, int num_sms, cudaStream_t s,
                                    int64_t* rows) {
    // chunks of up to 16 steps are one sub-segment (one recomputation); longer ones take the
    // sweep with 4-step sub-segments that keep their stage points
    if (a.max_chunk > 16) {
        if (a.max_chunk > kLx2sSub * kLx2sMaxSub) return cudaErrorInvalidValue;
        return pp ? launch_lorenz_x2_kernel(adjoint_lorenz_x2s_kernel<true>, a, num_sms, s, rows)
                  : launch_lorenz_x2_kernel(adjoint_lorenz_x2s_kernel<false>, a, num_sms, s, rows);
    }
    switch (m) {
    case 4: return pp ? launch_lorenz_x2_one<true, 4>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 4>(a, num_sms, s, rows);
    case 8: return pp ? launch_lorenz_x2_one<true, 8>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 8>(a, num_sms, s, rows);
    case 16: return pp ? launch_lorenz_x2_one<true, 16>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 16>(a, num_sms, s, rows);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ff
