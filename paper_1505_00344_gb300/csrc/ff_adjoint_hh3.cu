// ff_adjoint_hh3.cu -- discrete adjoint of the three coupled HH neurons (Eq. 6-11),
// the lane-split staged sweep, standalone and batched, in a unit of its own so the
// adjoint compiles in parallel.
//
// Lane layout.  Lanes 3j, 3j + 1 and 3j + 2 of a warp (j < 10) form triple j and
// hold neurons 0, 1 and 2 of particles 2j and 2j + 1 of the warp's 20: each f32x2
// register carries one quantity of one neuron of the two particles (lane 0 of the
// register particle 2j).  So every neuron's arithmetic runs packed, where the
// one-particle-per-thread form ran neuron 2 on floats and held all fifteen
// components of four adjoint vectors per thread.  The neurons of a particle meet
// only through the synaptic variables: the sum of the three s (the right-hand side)
// and the sum of the three synaptic products (the adjoint of s) are exchanged in
// the triple by shuffles, in the order of HH3::f.  Lanes 30 and 31 run on a copy of
// a valid particle and write nothing.
//
// Sweep.  Per chunk (in reverse): the chunk is recomputed once from its
// checkpoint with the integrator's own packed step (hh_neuron over f32x2, the bits
// of the taped forward), every RK4 step's four stage points (Euler: its state)
// going to the lane's scratch column in global memory; then the reverse steps run
// from last to first, each on stage points that cp.async copies brought into the
// lane's shared-memory column while the step before ran, and apply the four
// vector-Jacobian products, hand-differentiated from Eq. 6-11.
// The parameter gradient is carried in thirteen FP32 sums per neuron and particle
// over the chunk, from which the sixteen components are formed in FP64 at the
// chunk's end (each a sum times a parameter constant); the FP64 sums are reduced
// over particles through per-block partials in a fixed order.
#include "ff_adjoint_impl.cuh"

namespace ff {
namespace {

constexpr int kTriples = 10;                                   // lane triples per warp
constexpr int kWarpParticles = 2 * kTriples;                   // particles per warp
constexpr int kSplitBlock = 128;                               // threads per block
constexpr int kSplitBlockParticles = kSplitBlock / 32 * kWarpParticles;  // 80: one batched tile
// 3 blocks per SM leave 168 registers a thread: no spill (at 4 blocks the 128-register
// bound spilled, and keeping the parameter sums in shared memory instead cost more time)
constexpr int kSplitMinBlocks = 3;
constexpr int kStepPoints = 4 * 5;  // f32x2 entries of one RK4 step's stage points (4 points x 5 components)
static_assert(kSplitBlockParticles == kAdjTileHH3, "one batched tile per block");

__device__ __forceinline__ f2 mulp(f2 a, f2 b) { return mul2(a, b); }
__device__ __forceinline__ f2 kp(float c) { return pack2(c, c); }

__device__ __forceinline__ f2 lane_shfl(f2 v, int src) {
    f2 r;
    r.v = __shfl_sync(0xffffffffu, v.v, src);
    return r;
}

// (v of neuron 0 + v of neuron 1) + v of neuron 2 over the lane's triple, the order of
// HH3::f's sum of s.  src0 is the triple's first lane (lanes 30 and 31 read lanes 30, 31
// and 0: whatever they get is discarded).
__device__ __forceinline__ f2 triple_sum(f2 v, int src0) {
    const f2 a = lane_shfl(v, src0), b = lane_shfl(v, src0 + 1), c = lane_shfl(v, src0 + 2);
    return add2(add2(a, b), c);
}

// 8-byte asynchronous copy global -> shared (the issuing thread reads the copy after
// cp_async_wait), and the group boundaries of such copies.
__device__ __forceinline__ void cp_async8(unsigned long long* dst, const unsigned long long* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Per-lane constants of one chunk: the forward right-hand side's (hh_const per
// particle, as the two-particle integrator forms them: conductances and drive
// divided by C), the few more the products use, and the step sizes of the two
// particles.  The products run on the same C-divided conductances, so the factor
// 1 / C of the parameter gradients is applied once per chunk, in FP64.
struct LaneC {
    HHConst<HHPair> c;  // forward right-hand side
    f2 driveC;          // the lane's neuron drive / C (hh_drive_c)
    f2 sig, gNa3C, gK4C;  // sigma, 3 g_Na / C, 4 g_K / C
    f2 H1, H2, H6;      // h, h / 2, h / 6
};

__device__ __forceinline__ void lane_consts(LaneC& L, const float* pa, const float* pb, int n, float ha, float hb) {
    L.c = hh_const_pair(pa, pb);
    L.driveC = pack2(hh_drive_c(pa, n), hh_drive_c(pb, n));
    L.sig = pack2(pa[14], pb[14]);
    L.gNa3C = mulp(kp(3.0f), L.c.gNaC);
    L.gK4C = mulp(kp(4.0f), L.c.gKC);
    L.H1 = pack2(ha, hb);
    L.H2 = pack2(0.5f * ha, 0.5f * hb);
    L.H6 = pack2(ha * (1.0f / 6.0f), hb * (1.0f / 6.0f));
}

// One forward step of the lane's neuron (RK4 or Euler) from X, with its stage points
// written to out (f32x2 entries T apart: point s, component k at out[(s * 5 + k) * T];
// Euler: the state only).  Per lane of each register the operations of the
// integrator's steppers, so the recomputed states and stage points are the taped
// forward's.
template <int METHOD>
__device__ __forceinline__ void lane_fwd(f2 (&X)[5], const LaneC& L, int src0, unsigned long long* out, int64_t T) {
#pragma unroll
    for (int k = 0; k < 5; ++k) out[k * T] = X[k].v;
    if constexpr (METHOD == FF_EULER) {
        f2 K[5];
        hh_neuron<HHPair>(X[0], X[1], X[2], X[3], X[4], sub2(triple_sum(X[4], src0), X[4]), L.driveC, L.c, K);
#pragma unroll
        for (int k = 0; k < 5; ++k) X[k] = fma2(L.H1, K[k], X[k]);
    } else {
        f2 XS[5], A[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            XS[k] = X[k];
            A[k] = kp(0.0f);
        }
        // the four stages unrolled (so are the reverse step's four products): each lane
        // holds one neuron, so there is room for the next stage's independent work in flight
#pragma unroll
        for (int st = 0; st < 4; ++st) {
            f2 K[5];
            hh_neuron<HHPair>(XS[0], XS[1], XS[2], XS[3], XS[4], sub2(triple_sum(XS[4], src0), XS[4]), L.driveC, L.c,
                              K);
            const float w = (st == 1 || st == 2) ? 2.0f : 1.0f;  // fmaf(1, k, 0) = k
            const f2 W = kp(w);
#pragma unroll
            for (int k = 0; k < 5; ++k) A[k] = fma2(W, K[k], A[k]);
            if (st == 3) break;
            const f2 C = (st == 2) ? L.H1 : L.H2;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                XS[k] = fma2(C, K[k], X[k]);
                out[((st + 1) * 5 + k) * T] = XS[k].v;
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) X[k] = fma2(L.H6, A[k], X[k]);
    }
}

// FP32 sums over a chunk of one neuron lane's parameter contributions (v_V the
// adjoint of V, w_s = v_s (1 - s) / tau_r, a1 = act (1 - act), act the synaptic
// sigmoid), each with the factor that makes it a gradient component:
enum { A_U, A_CUR, A_NA, A_NAE, A_K, A_KE, A_L, A_SYN, A_SYNE, A_TR, A_TD, A_SG, A_TH, A_N };
struct LaneAcc {
    f2 r[A_N];
    __device__ __forceinline__ f2 get(int i) const { return r[i]; }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < A_N; ++i) r[i] = kp(0.0f);
    }
    __device__ __forceinline__ void add(int i, f2 x) { r[i] = add2(r[i], x); }
    __device__ __forceinline__ void fma(int i, f2 a, f2 b) { r[i] = fma2(a, b, r[i]); }
};

// One neuron lane's vector-Jacobian product at state x (others: the other two
// neurons' s), for input v = (v_V, v_m, v_h, v_n, v_s) of its components:
//   jx_V = sum over gates y of v_y (a_y' (1 - y) - b_y' y) + sigma a1 w_s - v_V g_tot / C
//   jx_y = (d I / d y) v_V / C - v_y (a_y + b_y)        for y = m, h, n
//   self = -v_s (act / tau_r + 1 / tau_d)                the own-s part of jx_s
//   syn  = g_syn (E_syn - V) v_V / C                      added to the other neurons' jx_s
// with the rates of the forward right-hand side, and the parameter sums added to acc.
__device__ __forceinline__ void lane_vjp(const f2 (&x)[5], f2 others, const f2 (&v)[5], const LaneC& L, f2 (&jx)[4],
                                         f2& self, f2& syn, LaneAcc& acc) {
    using O = HHPair;
    constexpr float kE25 = 12.182493960703473f;  // e^2.5
    constexpr float kE1 = 2.718281828459045f;    // e^1
    constexpr float kE3 = 20.085536923187668f;   // e^3
    constexpr float kQ = -kLog2e / 80.0f, kQ0 = 65.0f * (-kLog2e / 80.0f);
    constexpr float kB = -kLog2e / 18.0f, kB0 = 65.0f * (-kLog2e / 18.0f) + 2.0f;
    const f2 V = x[0], m = x[1], h = x[2], n = x[3], s = x[4];
    const f2 one = kp(1.0f);
    // rates and their derivatives
    const f2 q = O::ex2(fma2(V, kp(kQ), kp(kQ0)));
    const f2 q2 = mulp(q, q), q4 = mulp(q2, q2), q8 = mulp(q4, q4);
    const f2 bm = O::ex2(fma2(V, kp(kB), kp(kB0)));
    const f2 ah = mulp(kp(0.07f), q4);
    const f2 bn = mulp(kp(0.125f), q);
    const f2 es = O::ex2(fma2(L.c.neg_sig2, V, L.c.sig2_theta));
    const f2 ym = fma2(V, kp(0.1f), kp(4.0f)), yn = fma2(V, kp(0.1f), kp(5.5f));
    const auto sm = O::small(ym), sn = O::small(yn);
    const f2 em = mulp(kp(kE25), q8), en = mulp(kp(kE1), q8);
    const f2 dm = O::sel(sm, one, sub2(one, em)), dn = O::sel(sn, one, sub2(one, en));
    const f2 rmn = O::rcp(mulp(dm, dn));
    const f2 rm = mulp(dn, rmn), rn = mulp(dm, rmn);  // 1 / dm, 1 / dn
    // g(y) = y r with r = 1 / (1 - e^-y), and g'(y) = (1 - e^-y - y e^-y) r^2 = r (1 - e^-y g);
    // alpha_m = g(ym), alpha_n = g(yn) / 10; at most one of ym, yn lies in the series band
    const f2 ys = O::sel(sm, ym, yn);
    const f2 ser = bernoulli_series_t<O>(ys), dser = bernoulli_series_deriv_t<O>(ys);
    const f2 gmc = mulp(ym, rm), gnc = mulp(yn, rn);  // the closed forms
    const f2 am = O::sel(sm, ser, gmc);
    const f2 gn = O::sel(sn, ser, gnc);
    const f2 dgm = O::sel(sm, dser, mulp(O::fms(em, gmc, one), rm));
    const f2 dgn = O::sel(sn, dser, mulp(O::fms(en, gnc, one), rn));
    const f2 anbn = fma2(kp(0.1f), gn, bn);
    const f2 dam = mulp(kp(0.1f), dgm), dan = mulp(kp(0.01f), dgn);
    const f2 ph = fma2(kp(kE3), q8, one), ps = add2(one, es);
    const f2 r = O::rcp(mulp(ph, ps));
    const f2 bh = mulp(ps, r), act = mulp(ph, r);
    const f2 a1 = mulp(act, sub2(one, act));
    // minus the beta derivatives: beta_m' = -beta_m/18, beta_n' = -beta_n/80, beta_h' = beta_h (1 - beta_h)/10
    const f2 nd_bm = mulp(bm, kp(1.0f / 18.0f)), nd_bn = mulp(bn, kp(1.0f / 80.0f));
    const f2 nd_bh = mulp(mulp(kp(0.1f), bh), sub2(bh, one));
    const f2 dah = mulp(ah, kp(-1.0f / 20.0f));
    // currents and conductances, divided by C
    const f2 m2 = mulp(m, m), m3 = mulp(m2, m), m3h = mulp(m3, h);
    const f2 n2 = mulp(n, n), n3 = mulp(n2, n), n4 = mulp(n2, n2);
    const f2 dNa = sub2(L.c.ENa, V), dK = sub2(L.c.EK, V), dL = sub2(L.c.EL, V), dS = sub2(L.c.Esyn, V);
    const f2 gna = mulp(L.c.gNaC, m3h), gk = mulp(L.c.gKC, n4), gs = mulp(L.c.gsynC, others);
    f2 I = fma2(L.c.gLC, dL, L.driveC);
    I = fma2(gna, dNa, I);
    I = fma2(gk, dK, I);
    I = fma2(gs, dS, I);
    const f2 gtot = add2(gs, add2(gk, add2(gna, L.c.gLC)));
    // state
    const f2 vV = v[0];
    const f2 ws = mulp(mulp(v[4], L.c.inv_tr), sub2(one, s));  // v_s (1 - s) / tau_r
    // a' (1 - y) - b' y = a' + y (-b' - a')
    const f2 gate_m = fma2(m, sub2(nd_bm, dam), dam);
    const f2 gate_h = fma2(h, sub2(nd_bh, dah), dah);
    const f2 gate_n = fma2(n, sub2(nd_bn, dan), dan);
    const f2 a1ws = mulp(a1, ws);
    const f2 jv = fma2(v[1], gate_m, fma2(v[2], gate_h, fma2(v[3], gate_n, mulp(L.sig, a1ws))));
    jx[0] = O::fms(vV, gtot, jv);
    const f2 wNa = mulp(vV, dNa);
    jx[1] = O::fms(v[1], add2(am, bm), mulp(mulp(mulp(L.gNa3C, m2), h), wNa));
    jx[2] = O::fms(v[2], add2(ah, bh), mulp(mulp(L.c.gNaC, m3), wNa));
    jx[3] = O::fms(v[3], anbn, mulp(mulp(mulp(L.gK4C, n3), dK), vV));
    self = mulp(v[4], O::fms(act, L.c.inv_tr, L.c.neg_inv_td));  // -v_s (act / tau_r + 1 / tau_d)
    syn = mulp(mulp(L.c.gsynC, dS), vV);
    // parameter sums
    acc.add(A_U, vV);
    acc.fma(A_CUR, I, vV);
    const f2 tna = mulp(m3h, vV), tk = mulp(n4, vV), ts = mulp(others, vV);
    acc.add(A_NAE, tna);
    acc.fma(A_NA, tna, dNa);
    acc.add(A_KE, tk);
    acc.fma(A_K, tk, dK);
    acc.fma(A_L, dL, vV);
    acc.add(A_SYNE, ts);
    acc.fma(A_SYN, ts, dS);
    acc.fma(A_TR, act, ws);
    acc.fma(A_TD, s, v[4]);
    acc.add(A_TH, a1ws);
    acc.fma(A_SG, a1ws, V);
}

// The product at stage point x (others from the triple's s sum at it) and the full
// adjoint of the lane's components: jx_s gains the other two neurons' synaptic terms,
// (syn0 + syn1) + syn2 - syn_own.
__device__ __forceinline__ void lane_product(const f2 (&x)[5], f2 s_sum, const f2 (&v)[5], const LaneC& L, f2 (&out)[5],
                                             LaneAcc& acc, int src0) {
    f2 jx[4], self, syn;
    lane_vjp(x, sub2(s_sum, x[4]), v, L, jx, self, syn, acc);
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = jx[k];
    out[4] = add2(self, sub2(triple_sum(syn, src0), syn));
}

// Reverse of one RK4 step of the lane's neuron, from its stage points x1 = x,
// x2 = x + h/2 k1, x3 = x + h/2 k2, x4 = x + h k3 (pts: the lane's shared-memory
// column, stride bs, point s and component k at pts[(s * 5 + k) * bs]):
//   l4 = h/6 lam, l3 = h/3 lam + h m4, l2 = h/3 lam + h/2 m3, l1 = h/6 lam + h/2 m2
//   with m_s = J(x_s)^T l_s, and lam <- lam + ((m4 + m3) + m2) + m1.
__device__ __forceinline__ void lane_adj_rk4(const unsigned long long* pts, int bs, f2 (&lam)[5], const LaneC& L,
                                             LaneAcc& acc, int src0) {
    const f2 H3 = mulp(L.H1, kp(1.0f / 3.0f));
    f2 l[5], m[5], sum[5];
    // unrolled: a product's rate terms do not depend on the product before it, so they
    // overlap it (rolled, the sweep ran 14% slower)
#pragma unroll
    for (int st = 3; st >= 0; --st) {
        if (st == 3) {
#pragma unroll
            for (int k = 0; k < 5; ++k) l[k] = mulp(L.H6, lam[k]);
        } else {
            const f2 CL = (st == 0) ? L.H6 : H3, CM = (st == 2) ? L.H1 : L.H2;
#pragma unroll
            for (int k = 0; k < 5; ++k) l[k] = fma2(CL, lam[k], mulp(CM, m[k]));
        }
        f2 xs[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) xs[k].v = pts[(st * 5 + k) * bs];
        lane_product(xs, triple_sum(xs[4], src0), l, L, m, acc, src0);
        if (st == 3) {
#pragma unroll
            for (int k = 0; k < 5; ++k) sum[k] = m[k];
        } else if (st > 0) {
#pragma unroll
            for (int k = 0; k < 5; ++k) sum[k] = add2(sum[k], m[k]);
        }
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) lam[k] = add2(lam[k], add2(sum[k], m[k]));
}

// Reverse of one Euler step at state X: lam <- lam + J(X)^T (h lam).
__device__ __forceinline__ void lane_adj_euler(const f2 (&X)[5], f2 (&lam)[5], const LaneC& L, LaneAcc& acc,
                                               int src0) {
    f2 l[5], m[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) l[k] = mulp(L.H1, lam[k]);
    lane_product(X, triple_sum(X[4], src0), l, L, m, acc, src0);
#pragma unroll
    for (int k = 0; k < 5; ++k) lam[k] = add2(lam[k], m[k]);
}

// The lane's parameter vector for particle i (the per-particle parameter in place).
template <bool PP>
__device__ __forceinline__ void lane_params(const AdjointArgs& a, const AdjChunk& ch, int64_t i, float (&p)[HH3::NP]) {
    const float pv = PP ? a.pparam[i] : 0.0f;
#pragma unroll
    for (int q = 0; q < HH3::NP; ++q) p[q] = (PP && q == a.pidx) ? pv : ch.p[q];
}

__device__ __forceinline__ float group_h(const AdjointArgs& a, const AdjChunk& ch, int64_t i) {
    float h = ch.gh[0];
#pragma unroll
    for (int q = 1; q < FF_MAX_GROUPS; ++q)
        if (q < a.n_groups && i >= a.gstart[q]) h = ch.gh[q];
    return h;
}

// The sixteen parameter components of one particle's chunk sums (one lane of each
// register of acc), added to gacc (FP64).
__device__ __forceinline__ void add_chunk_grads(const float (&p)[HH3::NP], int n, float u, float cur, float na,
                                                float na_e, float k, float k_e, float l, float syn, float syn_e,
                                                float tr, float td, float sg, float th, double* gacc, int bs) {
    const double invC = 1.0 / (double)p[0], inv_tr = 1.0 / (double)p[12], inv_td = 1.0 / (double)p[13];
    double g[HH3::NP];
    g[0] = -(double)cur * invC;
    g[1] = (double)na * invC;
    g[2] = (double)k * invC;
    g[3] = (double)l * invC;
    g[4] = (double)p[1] * invC * (double)na_e;
    g[5] = (double)p[2] * invC * (double)k_e;
    g[6] = (double)p[3] * invC * (double)u;
    g[7] = (double)syn * invC;
    g[8] = (double)p[7] * invC * (double)syn_e;
    g[9] = n == 0 ? (double)u * invC : 0.0;
    g[10] = n == 1 ? (double)u * invC : 0.0;
    g[11] = n == 2 ? (double)u * invC : 0.0;
    g[12] = -(double)tr * inv_tr;
    g[13] = (double)td * inv_td * inv_td;
    g[14] = (double)sg - (double)p[15] * (double)th;
    g[15] = -(double)p[14] * (double)th;
#pragma unroll
    for (int q = 0; q < HH3::NP; ++q) gacc[q * bs] += g[q];
}

// Reverse sweep of one warp's particles [first, first + 20) clipped to end, over all
// chunks.  scr: the lane's scratch column (f32x2 entries T apart); stage and gacc:
// the lane's shared-memory columns (stride bs).  Every lane of the warp runs it whole
// (the shuffles need all 32); lanes without a particle compute on a copy of one and
// write nothing.
template <int METHOD, bool PP>
__device__ __forceinline__ void lane_sweep(const AdjointArgs& a, int64_t first, int64_t end,
                                           unsigned long long* scr, int64_t T, unsigned long long* stage,
                                           double* gacc, int bs) {
    constexpr int kPer = (METHOD == FF_EULER) ? 5 : kStepPoints;  // scratch entries per step
    const int lane = threadIdx.x & 31;
    const int j = lane / 3, n = lane - 3 * j, src0 = 3 * j;
    const int64_t i0 = first + 2 * j, i1 = i0 + 1;
    const bool v0 = j < kTriples && i0 < end, v1 = j < kTriples && i1 < end;
    const int64_t c0 = v0 ? i0 : first, c1 = v1 ? i1 : (v0 ? i0 : first);  // a valid particle to compute on
    f2 lam[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int64_t row = (int64_t)(5 * n + k) * a.n;
        lam[k] = pack2(a.lam_in[row + c0], a.lam_in[row + c1]);
    }
    for (int c = a.n_chunks - 1; c >= 0; --c) {
        const AdjChunk& ch = a.chunks[c];
        LaneC L;
        {
            float pa[HH3::NP], pb[HH3::NP];
            lane_params<PP>(a, ch, c0, pa);
            lane_params<PP>(a, ch, c1, pb);
            lane_consts(L, pa, pb, n, group_h(a, ch, c0), group_h(a, ch, c1));
        }
        const int Ls = ch.n_steps;
        const float* ck = a.ckpt + (int64_t)ch.ckpt * a.dim * a.pitch;
        f2 X[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float* plane = ck + (int64_t)(5 * n + k) * a.pitch;
            X[k] = pack2(plane[c0], plane[c1]);
        }
        // the chunk's recomputation: every step's stage points (Euler: states) to the scratch
#pragma unroll 1
        for (int r = 0; r < Ls; ++r) lane_fwd<METHOD>(X, L, src0, scr + (int64_t)r * kPer * T, T);
        LaneAcc acc;
        acc.zero();
        if constexpr (METHOD == FF_EULER) {
            // each step's state is loaded one step ahead, so the load's latency overlaps a step
            f2 Xn[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) Xn[k].v = scr[((int64_t)(Ls - 1) * 5 + k) * T];
#pragma unroll 1
            for (int r = Ls - 1; r >= 0; --r) {
#pragma unroll
                for (int k = 0; k < 5; ++k) X[k] = Xn[k];
                if (r > 0) {
#pragma unroll
                    for (int k = 0; k < 5; ++k) Xn[k].v = scr[((int64_t)(r - 1) * 5 + k) * T];
                }
                lane_adj_euler(X, lam, L, acc, src0);
            }
        } else {
            // a step's 20 stage-point entries are copied into one half of the lane's
            // shared-memory column while the step after it (in reverse) runs on the other
            auto fetch = [&](int r, int half) {
                const unsigned long long* src = scr + (int64_t)r * kStepPoints * T;
                unsigned long long* dst = stage + half * kStepPoints * bs;
#pragma unroll
                for (int q = 0; q < kStepPoints; ++q) cp_async8(dst + q * bs, src + q * T);
                cp_async_commit();
            };
            fetch(Ls - 1, 0);
#pragma unroll 1
            for (int r = Ls - 1, half = 0; r >= 0; --r, half ^= 1) {
                if (r > 0) fetch(r - 1, half ^ 1);
                else cp_async_commit();  // an empty group: the wait below still leaves step r's copies done
                cp_async_wait1();
                lane_adj_rk4(stage + half * kStepPoints * bs, bs, lam, L, acc, src0);
            }
        }
        float u[2], cur[2], na[2], na_e[2], kk[2], k_e[2], l[2], syn[2], syn_e[2], tr[2], td[2], sg[2], th[2];
        unpack2(acc.get(A_U), u[0], u[1]);
        unpack2(acc.get(A_CUR), cur[0], cur[1]);
        unpack2(acc.get(A_NA), na[0], na[1]);
        unpack2(acc.get(A_NAE), na_e[0], na_e[1]);
        unpack2(acc.get(A_K), kk[0], kk[1]);
        unpack2(acc.get(A_KE), k_e[0], k_e[1]);
        unpack2(acc.get(A_L), l[0], l[1]);
        unpack2(acc.get(A_SYN), syn[0], syn[1]);
        unpack2(acc.get(A_SYNE), syn_e[0], syn_e[1]);
        unpack2(acc.get(A_TR), tr[0], tr[1]);
        unpack2(acc.get(A_TD), td[0], td[1]);
        unpack2(acc.get(A_SG), sg[0], sg[1]);
        unpack2(acc.get(A_TH), th[0], th[1]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            if (e == 0 ? !v0 : !v1) continue;
            float p[HH3::NP];
            lane_params<PP>(a, ch, e == 0 ? i0 : i1, p);
            add_chunk_grads(p, n, u[e], cur[e], na[e], na_e[e], kk[e], k_e[e], l[e], syn[e], syn_e[e], tr[e], td[e],
                            sg[e], th[e], gacc, bs);
        }
    }
    float o0[5], o1[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) unpack2(lam[k], o0[k], o1[k]);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int64_t row = (int64_t)(5 * n + k) * a.n;
        if (v0) a.lam_out[row + i0] = o0[k];
        if (v1) a.lam_out[row + i1] = o1[k];
    }
}

// Shared memory of a block: the stage points and FP64 parameter sums of every lane.
struct SplitShared {
    unsigned long long stage[2 * kStepPoints * kSplitBlock];  // two steps' stage points per lane
    double gacc[HH3::NP * kSplitBlock];
    double red[kSplitBlock / 32][HH3::NP];
};

__device__ __forceinline__ void gacc_clear(SplitShared& sh) {
#pragma unroll
    for (int q = 0; q < HH3::NP; ++q) sh.gacc[q * kSplitBlock + threadIdx.x] = 0.0;
}

__device__ __forceinline__ void gacc_store(SplitShared& sh, double* row) {
    double g[HH3::NP];
#pragma unroll
    for (int q = 0; q < HH3::NP; ++q) g[q] = sh.gacc[q * kSplitBlock + threadIdx.x];
    block_sum_to_row<HH3::NP, kSplitBlock / 32>(g, sh.red, row);
}

template <int METHOD, bool PP>
__global__ void __launch_bounds__(kSplitBlock, kSplitMinBlocks) adjoint_hh3_split_kernel(
    const __grid_constant__ AdjointArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SplitShared& sh = *reinterpret_cast<SplitShared*>(smem_raw);
    gacc_clear(sh);
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long* scr = reinterpret_cast<unsigned long long*>(a.scratch) + t;
    const int64_t n_tasks = (a.n + kWarpParticles - 1) / kWarpParticles;
    const int64_t warps = (int64_t)gridDim.x * (kSplitBlock / 32);
    for (int64_t w = (int64_t)blockIdx.x * (kSplitBlock / 32) + (threadIdx.x >> 5); w < n_tasks; w += warps)
        lane_sweep<METHOD, PP>(a, w * kWarpParticles, a.n, scr, T, sh.stage + threadIdx.x, sh.gacc + threadIdx.x,
                               kSplitBlock);
    gacc_store(sh, a.partial + (int64_t)blockIdx.x * a.np_stride);
}

// Batched form: tiles of up to 80 particles of one member, one tile per block at a time.
template <int METHOD, bool PP>
__global__ void __launch_bounds__(kSplitBlock, kSplitMinBlocks) batch_adjoint_hh3_split_kernel(
    const __grid_constant__ BatchAdjointArgs b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SplitShared& sh = *reinterpret_cast<SplitShared*>(smem_raw);
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long* scr = reinterpret_cast<unsigned long long*>(b.scratch) + t;
    for (int tile = blockIdx.x; tile < b.n_tiles; tile += gridDim.x) {
        const AdjTile tl = b.tiles[tile];
        const AdjointArgs& a = b.sys[tl.sys];
        gacc_clear(sh);
        const int64_t first = tl.first + (int64_t)(threadIdx.x >> 5) * kWarpParticles;
        const int64_t end = tl.first + tl.count;
        if (first < end)  // warp-uniform
            lane_sweep<METHOD, PP>(a, first, end, scr, T, sh.stage + threadIdx.x, sh.gacc + threadIdx.x,
                                   kSplitBlock);
        gacc_store(sh, b.partial + (int64_t)tile * b.np_stride);
    }
}

// Resident threads of a kernel: the most it launches, and the scratch it needs room for.
template <class Kernel>
int64_t split_threads(Kernel kernel, int num_sms) {
    int occ = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared) != cudaSuccess)
        return 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SplitShared)) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kSplitBlock, sizeof(SplitShared)) !=
            cudaSuccess ||
        occ < 1)
        return 0;
    return (int64_t)occ * num_sms * kSplitBlock;
}

template <int METHOD, bool PP>
cudaError_t launch_split(const AdjointArgs& a, int num_sms, cudaStream_t s, int64_t* rows) {
    auto kernel = adjoint_hh3_split_kernel<METHOD, PP>;
    const int64_t resident = split_threads(kernel, num_sms);
    if (resident < kSplitBlock) return cudaErrorInvalidConfiguration;
    int64_t cap = resident / kSplitBlock;
    // room in the scratch: adjoint_scratch_floats_per_step floats per thread and step
    if (cap > a.scratch_threads / kSplitBlock) cap = a.scratch_threads / kSplitBlock;
    if (cap > 8 * a.max_blocks) cap = 8 * a.max_blocks;  // rows of the partial-sum buffer (one per block)
    const int64_t need = (a.n + kSplitBlockParticles - 1) / kSplitBlockParticles;
    const int grid = (int)(need < cap ? need : cap);
    if (grid < 1 || !a.scratch) return cudaErrorInvalidConfiguration;
    kernel<<<grid, kSplitBlock, sizeof(SplitShared), s>>>(a);
    *rows = grid;
    return cudaGetLastError();
}

template <int METHOD, bool PP>
cudaError_t launch_batch_split(const BatchAdjointArgs& b, int num_sms, cudaStream_t s) {
    auto kernel = batch_adjoint_hh3_split_kernel<METHOD, PP>;
    const int64_t resident = split_threads(kernel, num_sms);
    if (resident < kSplitBlock) return cudaErrorInvalidConfiguration;
    int64_t cap = resident / kSplitBlock;
    if (cap > b.scratch_threads / kSplitBlock) cap = b.scratch_threads / kSplitBlock;
    const int grid = (int)((int64_t)b.n_tiles < cap ? b.n_tiles : cap);
    if (grid < 1) return cudaSuccess;
    if (!b.scratch) return cudaErrorInvalidConfiguration;
    kernel<<<grid, kSplitBlock, sizeof(SplitShared), s>>>(b);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint_hh3(int method, bool pp, int /*m*/, const AdjointArgs& a, int /*block*/, int num_sms,
                               cudaStream_t s, int64_t* rows) {
    if (method == FF_RK4)
        return pp ? launch_split<FF_RK4, true>(a, num_sms, s, rows) : launch_split<FF_RK4, false>(a, num_sms, s, rows);
    return pp ? launch_split<FF_EULER, true>(a, num_sms, s, rows) : launch_split<FF_EULER, false>(a, num_sms, s, rows);
}

cudaError_t launch_batch_adjoint_hh3(int method, bool pp, int /*m*/, const BatchAdjointArgs& b, int num_sms,
                                     cudaStream_t s) {
    if (method == FF_RK4)
        return pp ? launch_batch_split<FF_RK4, true>(b, num_sms, s) : launch_batch_split<FF_RK4, false>(b, num_sms, s);
    return pp ? launch_batch_split<FF_EULER, true>(b, num_sms, s) : launch_batch_split<FF_EULER, false>(b, num_sms, s);
}

int64_t adjoint_scratch_threads_hh3(int method, bool pp, int num_sms, bool batched) {
    if (batched) {
        if (method == FF_RK4)
            return pp ? split_threads(batch_adjoint_hh3_split_kernel<FF_RK4, true>, num_sms)
                      : split_threads(batch_adjoint_hh3_split_kernel<FF_RK4, false>, num_sms);
        return pp ? split_threads(batch_adjoint_hh3_split_kernel<FF_EULER, true>, num_sms)
                  : split_threads(batch_adjoint_hh3_split_kernel<FF_EULER, false>, num_sms);
    }
    if (method == FF_RK4)
        return pp ? split_threads(adjoint_hh3_split_kernel<FF_RK4, true>, num_sms)
                  : split_threads(adjoint_hh3_split_kernel<FF_RK4, false>, num_sms);
    return pp ? split_threads(adjoint_hh3_split_kernel<FF_EULER, true>, num_sms)
              : split_threads(adjoint_hh3_split_kernel<FF_EULER, false>, num_sms);
}

}  // namespace ff
