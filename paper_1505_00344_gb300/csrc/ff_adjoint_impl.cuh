// ff_adjoint_impl.cuh -- device code and launch templates of the discrete
// adjoint of the RK4 / Euler integrator (not part of the paper), shared by the
// per-family translation units (ff_adjoint_lorenz.cu, ff_adjoint_hh3.cu,
// ff_adjoint_small.cu, ff_adjoint_linear.cu), which compile in parallel.
//
// One thread per particle walks the chunks in reverse with the adjoint state
// lambda = dL/dx in registers.  A chunk of L <= M*M steps is recomputed from its
// checkpoint twice (once when L <= M): once to place sub-checkpoints every M
// steps (local memory), then per sub-segment (in reverse) to put its <= M
// states in registers (local memory for the 15-dimensional system), which the
// reverse RK4 steps consume from last to first.  Parameter gradients are summed
// per particle in FP32 within a chunk, added to FP64 per chunk, and reduced
// over particles through per-block FP64 partials in fixed order.
#pragma once

#include <cstdint>
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
        const float SE = __fdividef(1.0f, 1.0f + exp2f(g2 * (th - aE)));
        const float SI = __fdividef(1.0f, 1.0f + exp2f(g2 * (th - aI)));
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

// g(y) = y / (1 - e^-y) and g'(y) = (1 - e^-y (1 + y)) / (1 - e^-y)^2, given e = e^-y.
// For |y| < 0.5, where the differences cancel in FP32, the Bernoulli series
// g' = 1/2 + y/6 - y^3/180 + y^5/5040 - y^7/151200 (next term below 1e-9).
__device__ __forceinline__ void x_over_expm1(float y, float e, float& g, float& dg) {
    if (fabsf(y) < 0.5f) {
        const float y2 = y * y;
        g = bernoulli_series(y);
        dg = fmaf(y, fmaf(y2, fmaf(y2, fmaf(y2, -1.0f / 151200.0f, 1.0f / 5040.0f), -1.0f / 180.0f), 1.0f / 6.0f),
                  0.5f);
    } else {
        const float r = __fdividef(1.0f, __fsub_rn(1.0f, e));
        g = y * r;
        dg = fmaf(-e, 1.0f + y, 1.0f) * r * r;
    }
}

template <> struct Vjp<HH3> {
    // Eq. 6-11 differentiated term by term; the gate rates depend on V only.
    // Per neuron i with u_i = v_V,i / C:
    //   d/dV_i: -u_i (gL + gNa m^3 h + gK n^4 + gsyn S_i) + sum over gates of
    //           v_y (a'(1 - y) - b' y) + v_s sig act (1 - act)(1 - s) / tau_r
    //   d/dm, d/dh, d/dn: the current terms' derivatives times u_i minus v_y (a + b)
    //   d/ds_i: -v_s (act / tau_r + 1 / tau_d) + sum_{j != i} gsyn (Esyn - V_j) u_j
    // where S_i is the sum of the other neurons' s.
    __device__ __forceinline__ static void apply(const float (&x)[15], const float* p, const float (&v)[15],
                                                 float (&jx)[15], float* jp) {
        const float C = p[0], gNa = p[1], gK = p[2], gL = p[3];
        const float ENa = p[4], EK = p[5], EL = p[6], gsyn = p[7], Esyn = p[8];
        const float inv_tr = __fdividef(1.0f, p[12]), inv_td = __fdividef(1.0f, p[13]);
        const float sig = p[14], theta = p[15];
        const float invC = __fdividef(1.0f, C);
        const float s_sum = x[4] + x[9] + x[14];
        constexpr float kE25 = 12.182493960703473f;  // e^2.5
        constexpr float kE1 = 2.718281828459045f;    // e^1
        constexpr float kE3 = 20.085536923187668f;   // e^3
        float syn[3], self_s[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float V = x[5 * i], m = x[5 * i + 1], h = x[5 * i + 2], n = x[5 * i + 3], s = x[5 * i + 4];
            const float uV = v[5 * i] * invC, vm = v[5 * i + 1], vh = v[5 * i + 2], vn = v[5 * i + 3];
            const float vs = v[5 * i + 4];
            // rates (same formulation as the forward right-hand side)
            const float u = V + 65.0f;
            const float q = exp2f(u * (-kLog2e / 80.0f));
            const float q2 = q * q, q4 = q2 * q2, q8 = q4 * q4;
            const float bm = 4.0f * exp2f(u * (-kLog2e / 18.0f));
            const float ah = 0.07f * q4;
            const float bn = 0.125f * q;
            const float bh = __fdividef(1.0f, fmaf(kE3, q8, 1.0f));
            const float act = __fdividef(1.0f, 1.0f + exp2f(sig * kLog2e * (theta - V)));
            float gm, dgm, gn, dgn;
            x_over_expm1((V + 40.0f) * 0.1f, kE25 * q8, gm, dgm);
            x_over_expm1((V + 55.0f) * 0.1f, kE1 * q8, gn, dgn);
            const float am = gm, dam = 0.1f * dgm;   // alpha_m = 0.1 (V+40) / (1 - e^{-(V+40)/10})
            const float an = 0.1f * gn, dan = 0.01f * dgn;
            const float dbm = bm * (-1.0f / 18.0f), dah = ah * (-1.0f / 20.0f), dbn = bn * (-1.0f / 80.0f);
            const float dbh = 0.1f * bh * (1.0f - bh);
            const float a1 = act * (1.0f - act);
            // currents
            const float m2 = m * m, m3 = m2 * m, m3h = m3 * h;
            const float n2 = n * n, n3 = n2 * n, n4 = n2 * n2;
            const float others = s_sum - s;
            const float dNa = ENa - V, dK = EK - V, dL = EL - V, dS = Esyn - V;
            float I = gL * dL;
            I = fmaf(gNa * m3h, dNa, I);
            I = fmaf(gK * n4, dK, I);
            I = fmaf(gsyn * others, dS, I);
            I = I + p[9 + i];
            const float gtot = fmaf(gsyn, others, fmaf(gK, n4, fmaf(gNa, m3h, gL)));
            float jv = -uV * gtot;
            jv = fmaf(vm, fmaf(dam, 1.0f - m, -dbm * m), jv);
            jv = fmaf(vh, fmaf(dah, 1.0f - h, -dbh * h), jv);
            jv = fmaf(vn, fmaf(dan, 1.0f - n, -dbn * n), jv);
            const float sv = vs * inv_tr * (1.0f - s);  // v_s (1 - s) / tau_r
            jv = fmaf(sig * a1, sv, jv);
            jx[5 * i] = jv;
            jx[5 * i + 1] = fmaf(uV * 3.0f * gNa * m2 * h, dNa, -vm * (am + bm));
            jx[5 * i + 2] = fmaf(uV * gNa * m3, dNa, -vh * (ah + bh));
            jx[5 * i + 3] = fmaf(uV * 4.0f * gK * n3, dK, -vn * (an + bn));
            self_s[i] = -vs * fmaf(act, inv_tr, inv_td);
            syn[i] = gsyn * dS * uV;
            // parameters
            jp[0] = fmaf(-I * invC, uV, jp[0]);
            jp[1] = fmaf(m3h * dNa, uV, jp[1]);
            jp[2] = fmaf(n4 * dK, uV, jp[2]);
            jp[3] = fmaf(dL, uV, jp[3]);
            jp[4] = fmaf(gNa * m3h, uV, jp[4]);
            jp[5] = fmaf(gK * n4, uV, jp[5]);
            jp[6] = fmaf(gL, uV, jp[6]);
            jp[7] = fmaf(dS * others, uV, jp[7]);
            jp[8] = fmaf(gsyn * others, uV, jp[8]);
            jp[9 + i] = __fadd_rn(jp[9 + i], uV);
            jp[12] = fmaf(-act * inv_tr, sv, jp[12]);
            jp[13] = fmaf(s * inv_td * inv_td, vs, jp[13]);
            jp[14] = fmaf(a1 * (V - theta), sv, jp[14]);
            jp[15] = fmaf(-sig * a1, sv, jp[15]);
        }
        const float syn_sum = syn[0] + syn[1] + syn[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) jx[5 * i + 4] = __fadd_rn(self_s[i], syn_sum - syn[i]);
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
    const float h2 = 0.5f * h, h6 = h * (1.0f / 6.0f);
    float k[D], xs[D], acc[D];
    if constexpr (D > 8) {
        // large systems: the forward integrator's own RK4 stepper (for HH3 the packed
        // neuron pairs), so the recomputed states are the taped forward's, bit for bit
        typename StepperFor<R, FF_RK4, false>::type st;
        float sc[D];
        st.init(h, p);
        st.acc(x, acc, sc);
#pragma unroll
        for (int i = 0; i < D; ++i) x[i] = fmaf(sc[i], acc[i], x[i]);
        return;
    }
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
    const float h2 = 0.5f * h, h3 = h * (1.0f / 3.0f), h6 = h * (1.0f / 6.0f);
    if constexpr (D > 8) {
        // large systems: stage points in a (local-memory) array, each pass one copy of f
        // or of the vector-Jacobian product; the same operations in the same order as below
        float xs[4][D], k[D], l[D], m[D], sum[D];
#pragma unroll
        for (int i = 0; i < D; ++i) xs[0][i] = x[i];
#pragma unroll 1
        for (int st = 0; st < 3; ++st) {
            R::f(xs[st], p, k);
            const float c = (st == 2) ? h : h2;
#pragma unroll
            for (int i = 0; i < D; ++i) xs[st + 1][i] = fmaf(c, k[i], x[i]);
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
            Vjp<R>::apply(xs[st], p, l, m, jp);
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
        return;
    }
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
// lam_out, parameter contributions added to gacc (FP64, per chunk).
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
            if constexpr (D > 8) {
                // large states: the sub-segment stays in local memory (indexed at run time)
                for (int r = 0; r < nq; ++r) {
#pragma unroll
                    for (int k = 0; k < D; ++k) st[r][k] = x[k];
                    if (r + 1 < nq) fwd_step<R, METHOD>(x, h, p);
                }
                for (int r = nq - 1; r >= 0; --r) adj_step<R, METHOD>(st[r], lam, h, p, jp);
            } else {
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
// Packed-pair adjoint for Lorenz RK4: two particles per thread in f32x2
// registers (lane 0 particle 2t, lane 1 particle 2t + 1).  Every operation is
// the scalar adjoint's, lane by lane (Lorenz::f, the RK4 step, Vjp<Lorenz> and
// the reverse step; negations as 0 - x, which is exact), so dL/dx0 is the same
// to the bit and the parameter sums differ only in their FP64 order.
// ---------------------------------------------------------------------------
__device__ __forceinline__ f2 neg2(f2 a) { return sub2(pack2(0.0f, 0.0f), a); }
__device__ __forceinline__ f2 mul2a(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
    return r;
}

struct LorenzPairP {
    f2 s, ns, r, nb;  // sigma, -sigma, r, -beta per lane
};

__device__ __forceinline__ void lorenz_f2(const f2 (&x)[3], const LorenzPairP& c, f2 (&k)[3]) {
    k[0] = mul2a(c.s, sub2(x[1], x[0]));
    k[1] = fma2(x[0], sub2(c.r, x[2]), neg2(x[1]));
    k[2] = fma2(x[0], x[1], mul2a(c.nb, x[2]));
}

__device__ __forceinline__ void lorenz_fwd2(f2 (&x)[3], f2 h, f2 h2, f2 h6, const LorenzPairP& c) {
    const f2 two = pack2(2.0f, 2.0f);
    f2 k[3], xs[3], acc[3];
    lorenz_f2(x, c, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) { acc[i] = k[i]; xs[i] = fma2(h2, k[i], x[i]); }
    lorenz_f2(xs, c, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) { acc[i] = fma2(two, k[i], acc[i]); xs[i] = fma2(h2, k[i], x[i]); }
    lorenz_f2(xs, c, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) { acc[i] = fma2(two, k[i], acc[i]); xs[i] = fma2(h, k[i], x[i]); }
    lorenz_f2(xs, c, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) x[i] = fma2(h6, add2(acc[i], k[i]), x[i]);
}

// jx = J(x)^T v, jp += F_p(x)^T v (Vjp<Lorenz> lane by lane)
__device__ __forceinline__ void lorenz_vjp2(const f2 (&x)[3], const LorenzPairP& c, const f2 (&v)[3], f2 (&jx)[3],
                                            f2 (&jp)[3]) {
    jx[0] = fma2(c.ns, v[0], fma2(sub2(c.r, x[2]), v[1], mul2a(x[1], v[2])));
    jx[1] = fma2(c.s, v[0], fma2(x[0], v[2], neg2(v[1])));
    jx[2] = fma2(neg2(x[0]), v[1], mul2a(c.nb, v[2]));
    jp[0] = fma2(sub2(x[1], x[0]), v[0], jp[0]);
    jp[1] = fma2(x[0], v[1], jp[1]);
    jp[2] = fma2(neg2(x[2]), v[2], jp[2]);
}

__device__ __forceinline__ void lorenz_adj2(const f2 (&x)[3], f2 (&lam)[3], f2 h, f2 h2, f2 h3, f2 h6,
                                            const LorenzPairP& c, f2 (&jp)[3]) {
    f2 k[3], x2[3], x3[3], x4[3];
    lorenz_f2(x, c, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) x2[i] = fma2(h2, k[i], x[i]);
    lorenz_f2(x2, c, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) x3[i] = fma2(h2, k[i], x[i]);
    lorenz_f2(x3, c, k);
#pragma unroll
    for (int i = 0; i < 3; ++i) x4[i] = fma2(h, k[i], x[i]);
    f2 l[3], m[3], sum[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) l[i] = mul2a(h6, lam[i]);
    lorenz_vjp2(x4, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = m[i]; l[i] = fma2(h3, lam[i], mul2a(h, m[i])); }
    lorenz_vjp2(x3, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = add2(sum[i], m[i]); l[i] = fma2(h3, lam[i], mul2a(h2, m[i])); }
    lorenz_vjp2(x2, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) { sum[i] = add2(sum[i], m[i]); l[i] = fma2(h6, lam[i], mul2a(h2, m[i])); }
    lorenz_vjp2(x, c, l, m, jp);
#pragma unroll
    for (int i = 0; i < 3; ++i) lam[i] = add2(lam[i], add2(sum[i], m[i]));
}

template <bool PP, int M>
__global__ void __launch_bounds__(128, 3) adjoint_lorenz_x2_kernel(const __grid_constant__ AdjointArgs a) {
    __shared__ double red[4][3];
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
            LorenzPairP cp2;
            cp2.s = pack2(pa[0], pb[0]);
            cp2.ns = pack2(-pa[0], -pb[0]);
            cp2.r = pack2(pa[1], pb[1]);
            cp2.nb = pack2(-pa[2], -pb[2]);
            const float ha = ch.gh[g0], hb = ch.gh[g1];
            const f2 h = pack2(ha, hb), h2 = pack2(0.5f * ha, 0.5f * hb);
            const f2 h3 = pack2(ha * (1.0f / 3.0f), hb * (1.0f / 3.0f)), h6 = pack2(ha * (1.0f / 6.0f), hb * (1.0f / 6.0f));
            const int L = ch.n_steps;
            const float* ck = a.ckpt + (int64_t)ch.ckpt * a.dim * a.pitch;
            f2 x[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) x[k] = pack2(ck[k * a.pitch + i0], ck[k * a.pitch + i1]);  // pitch covers i1
            f2 cpt[M][3];
            int nsub = 0;
            for (int base = 0; base < L; base += M, ++nsub) {
#pragma unroll
                for (int k = 0; k < 3; ++k) cpt[nsub][k] = x[k];
                const int nq = (base + M < L) ? M : 0;
#pragma unroll 1
                for (int r = 0; r < nq; ++r) lorenz_fwd2(x, h, h2, h6, cp2);
            }
            f2 jp[3] = {pack2(0.f, 0.f), pack2(0.f, 0.f), pack2(0.f, 0.f)};
            for (int sq = nsub - 1; sq >= 0; --sq) {
                const int nq = min(M, L - sq * M);
                f2 st[M][3];
#pragma unroll
                for (int k = 0; k < 3; ++k) x[k] = cpt[sq][k];
#pragma unroll
                for (int r = 0; r < M; ++r) {
                    if (r < nq) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) st[r][k] = x[k];
                        if (r + 1 < nq) lorenz_fwd2(x, h, h2, h6, cp2);
                    }
                }
#pragma unroll
                for (int r = M - 1; r >= 0; --r)
                    if (r < nq) lorenz_adj2(st[r], lam, h, h2, h3, h6, cp2, jp);
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
    block_sum_to_row<3, 4>(gacc, red, a.partial + (int64_t)blockIdx.x * a.np_stride);
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

template <bool PP, int M>
static cudaError_t launch_lorenz_x2_one(const AdjointArgs& a, int num_sms, cudaStream_t s, int64_t* rows) {
    auto kernel = adjoint_lorenz_x2_kernel<PP, M>;
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 128, 0);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int64_t need = ((a.n + 1) / 2 + 127) / 128;
    int64_t cap = (int64_t)occ * num_sms;
    if (cap > a.max_blocks) cap = a.max_blocks;  // rows of the partial-sum buffer
    const int grid = (int)(need < cap ? need : cap);
    if (grid < 1) return cudaErrorInvalidConfiguration;
    kernel<<<grid, 128, 0, s>>>(a);
    *rows = grid;
    return cudaGetLastError();
}

static cudaError_t launch_lorenz_x2(bool pp, int m, const AdjointArgs& a, int num_sms, cudaStream_t s,
                                    int64_t* rows) {
    switch (m) {
    case 4: return pp ? launch_lorenz_x2_one<true, 4>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 4>(a, num_sms, s, rows);
    case 8: return pp ? launch_lorenz_x2_one<true, 8>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 8>(a, num_sms, s, rows);
    case 16: return pp ? launch_lorenz_x2_one<true, 16>(a, num_sms, s, rows) : launch_lorenz_x2_one<false, 16>(a, num_sms, s, rows);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace ff
