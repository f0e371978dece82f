/*
 * ffo.c -- plain, slow, single-threaded FP64 oracle for the Fireflies hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm load it.  It shares no source, header, table or helper with the CUDA
 * library; the two meet only through inputs produced by the seeded workload
 * generators.
 *
 * Compile with -O2 -ffp-contract=off (no fused multiply-add anywhere), so every
 * floating-point operation below rounds exactly where it is written.
 *
 * What is computed, in the paper's order and notation:
 *   - initial conditions drawn uniformly from each particle group's box
 *     (Appendix A, "Particle Group" and "Initialization"), with the counter-based
 *     SplitMix64 generator standing in for the paper's unspecified NumPy RNG;
 *   - the per-system right-hand sides: Wilson-Cowan form of Eq. 1-2, Lorenz
 *     Eq. 3-5, three coupled Hodgkin-Huxley neurons Eq. 6-11 (all-to-all
 *     inhibitory coupling and modern-convention constants, per the measured
 *     workload), plus two linear test systems;
 *   - classical fourth-order Runge-Kutta with a constant step (Sec. 2.1, and
 *     Appendix A "Initialization": read position, RK4 update, write back) and
 *     the explicit Euler step;
 *   - backward-time groups as a negative step (Appendix A, "Running the
 *     Simulation");
 *   - per-particle parameter values for dynamic bifurcation diagrams (Sec. 2.1
 *     last paragraph, Sec. 2.2 last paragraph): the parameter becomes a state
 *     variable with zero derivative, whose initial values form a linspace;
 *   - projection of each state to the screen (Appendix A, vertex and geometry
 *     shaders: 2D window map, or 4x4 Model-View-Projection with perspective
 *     divide) and additive point splatting into a count image (fragment
 *     shader with GL_ONE blending).  Projection and pixel decisions are made in
 *     FP32, the precision the paper's render path works in, with every
 *     operation rounded separately.
 *
 * Every function here is pinned by a test in tests/test_oracle_*.py against a
 * closed form, a published value or a fact printed in the paper.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

#define FFO_MAXD 16

enum { FFO_LINEAR = 0, FFO_HARMONIC = 1, FFO_WILSON_COWAN = 2, FFO_LORENZ = 3, FFO_HH3 = 4 };
enum { FFO_RK4 = 0, FFO_EULER = 1 };

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number     */
/* generators", OOPSLA 2014; Vigna's public-domain splitmix64.c): the state   */
/* advances by the golden-ratio increment and each output is the state passed */
/* through the variant-13 finaliser.  Output n (n >= 1) of the stream seeded  */
/* with s is therefore mix(s + n * increment), which makes it counter based.  */
/* ------------------------------------------------------------------------ */
uint64_t ffo_splitmix64(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform initial conditions for particles of one group (Appendix A: each
 * group's initial-condition ranges define a box; each particle gets a
 * uniformly random point in it).  Particle j (index within its group) and
 * state variable k use draw n = j*dim + k + 1 of the group's stream; the top
 * 24 bits give u in [0,1); x = lo + (hi - lo) * u in double, then rounded to
 * the nearest float because the state array is single precision (Appendix A).
 * out is SoA: out[k * out_pitch + t] for t in [0, count).  If idx is not NULL
 * the t-th output particle is group particle idx[t], else j0 + t. */
void ffo_seed_group(int dim, int64_t count, int64_t j0, const int64_t *idx,
                    const double *lo, const double *hi, uint64_t seed,
                    float *out, int64_t out_pitch)
{
    for (int64_t t = 0; t < count; ++t) {
        int64_t j = idx ? idx[t] : j0 + t;
        for (int k = 0; k < dim; ++k) {
            uint64_t r = ffo_splitmix64(seed, (uint64_t)j * (uint64_t)dim + (uint64_t)k + 1u);
            double u = (double)(r >> 40) * (1.0 / 16777216.0);
            double width = hi[k] - lo[k];
            double x = lo[k] + width * u;
            out[(int64_t)k * out_pitch + t] = (float)x;
        }
    }
}

/* Per-particle bifurcation parameter: particle i of P gets
 * lo + (hi - lo) * (i / (P - 1)) in double, rounded to float because the
 * paper stores it as an extra single-precision state variable with zero time
 * derivative (Sec. 2.1, last paragraph).  P == 1 gives lo. */
void ffo_linspace(int64_t P, int64_t i0, int64_t count, const int64_t *idx,
                  double lo, double hi, float *out)
{
    for (int64_t t = 0; t < count; ++t) {
        int64_t i = idx ? idx[t] : i0 + t;
        double frac = (P > 1) ? (double)i / (double)(P - 1) : 0.0;
        double width = hi - lo;
        out[t] = (float)(lo + width * frac);
    }
}

/* ------------------------------------------------------------------------ */
/* Right-hand sides f(x, p).                                                  */
/* ------------------------------------------------------------------------ */

/* Linear test system dx/dt = A x, A row-major dim x dim in p. */
static void rhs_linear(int dim, const double *x, const double *p, double *dx)
{
    for (int i = 0; i < dim; ++i) {
        double s = 0.0;
        for (int j = 0; j < dim; ++j) s += p[i * dim + j] * x[j];
        dx[i] = s;
    }
}

/* Harmonic oscillator: dx/dt = v, dv/dt = -omega^2 x;  p = [omega]. */
static void rhs_harmonic(const double *x, const double *p, double *dx)
{
    double w = p[0];
    dx[0] = x[1];
    dx[1] = -(w * w) * x[0];
}

/* Logistic response curve of the Wilson-Cowan populations (the Z_s, Z_g of
 * Eq. 1-2): S(a) = 1 / (1 + exp(-gain * (a - threshold))). */
static double wc_sigmoid(double a, double gain, double thresh)
{
    return 1.0 / (1.0 + exp(-gain * (a - thresh)));
}

/* Wilson-Cowan E-I model, Eq. 1-2 with x = E (excitatory), y = I (inhibitory):
 *   tauE dE/dt = -E + S(wEE E - wEI I + P)
 *   tauI dI/dt = -I + S(wIE E - wII I + Q)
 * p = [wEE, wEI, wIE, wII, P, Q, tauE, tauI, gain, threshold]. */
static void rhs_wilson_cowan(const double *x, const double *p, double *dx)
{
    double E = x[0], I = x[1];
    double wEE = p[0], wEI = p[1], wIE = p[2], wII = p[3];
    double P = p[4], Q = p[5], tauE = p[6], tauI = p[7], gain = p[8], th = p[9];
    double aE = wEE * E - wEI * I + P;
    double aI = wIE * E - wII * I + Q;
    dx[0] = (-E + wc_sigmoid(aE, gain, th)) / tauE;
    dx[1] = (-I + wc_sigmoid(aI, gain, th)) / tauI;
}

/* Lorenz, Eq. 3-5:  dx = sigma (y - x),  dy = x (r - z) - y,  dz = x y - beta z.
 * p = [sigma, r, beta]. */
static void rhs_lorenz(const double *x, const double *p, double *dx)
{
    double sigma = p[0], r = p[1], beta = p[2];
    dx[0] = sigma * (x[1] - x[0]);
    dx[1] = x[0] * (r - x[2]) - x[1];
    dx[2] = x[0] * x[1] - beta * x[2];
}

/* v / (1 - exp(-v / 10)), the shape shared by alpha_m and alpha_n.  The
 * denominator is written with the C99 library primitive expm1, which keeps full
 * precision as v -> 0; at v = 0 exactly the quotient is 0/0 and takes its
 * limit 10. */
static double hh_vtrap(double v)
{
    if (v == 0.0) return 10.0;
    return v / (-expm1(-v / 10.0));
}

/* d/dv of v / (1 - e^(-v/10)).  With x = v/10 it is g'(x) for g(x) = x / (1 - e^-x),
 * g'(x) = (1 - e^-x (1 + x)) / (1 - e^-x)^2.  Near x = 0 the numerator cancels, so
 * there the Taylor series of g' (from g = 1 + x/2 + x^2/12 - x^4/720 + x^6/30240 - ...,
 * the Bernoulli-number expansion) is used: 1/2 + x/6 - x^3/180 + x^5/5040 - x^7/151200. */
static double hh_vtrap_deriv(double v)
{
    double x = v / 10.0;
    if (fabs(x) < 1e-2) {
        double x2 = x * x;
        return 0.5 + x * (1.0 / 6.0 + x2 * (-1.0 / 180.0 + x2 * (1.0 / 5040.0 - x2 / 151200.0)));
    }
    double e = exp(-x), d = -expm1(-x);
    return (1.0 - e * (1.0 + x)) / (d * d);
}

/* Hodgkin-Huxley rate functions of the squid axon (Hodgkin & Huxley 1952,
 * cited for Eq. 6-9) in the convention with rest near -65 mV. */
static double hh_alpha_m(double V) { return 0.1 * hh_vtrap(V + 40.0); }
static double hh_beta_m(double V)  { return 4.0 * exp(-(V + 65.0) / 18.0); }
static double hh_alpha_h(double V) { return 0.07 * exp(-(V + 65.0) / 20.0); }
static double hh_beta_h(double V)  { return 1.0 / (1.0 + exp(-(V + 35.0) / 10.0)); }
static double hh_alpha_n(double V) { return 0.01 * hh_vtrap(V + 55.0); }
static double hh_beta_n(double V)  { return 0.125 * exp(-(V + 65.0) / 80.0); }

/* Three coupled Hodgkin-Huxley neurons, Eq. 6-11.  Neuron i has state
 * (V_i, m_i, h_i, n_i, s_i) at x[5i .. 5i+4].
 *   C dV_i = gL (EL - V_i) + gNa m_i^3 h_i (ENa - V_i) + gK n_i^4 (EK - V_i)
 *            + I_syn,i + I_i                                          (Eq. 6)
 *   dh_i = alpha_h (1 - h_i) - beta_h h_i, same for m and n           (Eq. 7-9)
 *   I_syn,i = gsyn (Esyn - V_i) * sum_{j != i} s_j      (Eq. 10, all-to-all)
 *   ds_i = (1/tau_r) (1 + exp(-sig (V_i - theta)))^-1 (1 - s_i) - s_i / tau_d
 *                                                                      (Eq. 11)
 * p = [C, gNa, gK, gL, ENa, EK, EL, gsyn, Esyn, I1, I2, I3,
 *      tau_r, tau_d, sig, theta]. */
static void rhs_hh3(const double *x, const double *p, double *dx)
{
    double C = p[0], gNa = p[1], gK = p[2], gL = p[3];
    double ENa = p[4], EK = p[5], EL = p[6], gsyn = p[7], Esyn = p[8];
    double tau_r = p[12], tau_d = p[13], sig = p[14], theta = p[15];
    for (int i = 0; i < 3; ++i) {
        const double *xi = x + 5 * i;
        double V = xi[0], m = xi[1], h = xi[2], n = xi[3], s = xi[4];
        double s_others = 0.0;
        for (int j = 0; j < 3; ++j)
            if (j != i) s_others += x[5 * j + 4];
        double I_L = gL * (EL - V);
        double I_Na = gNa * (m * m * m) * h * (ENa - V);
        double I_K = gK * (n * n * n * n) * (EK - V);
        double I_syn = gsyn * (Esyn - V) * s_others;
        double *di = dx + 5 * i;
        di[0] = (I_L + I_Na + I_K + I_syn + p[9 + i]) / C;
        di[1] = hh_alpha_m(V) * (1.0 - m) - hh_beta_m(V) * m;
        di[2] = hh_alpha_h(V) * (1.0 - h) - hh_beta_h(V) * h;
        di[3] = hh_alpha_n(V) * (1.0 - n) - hh_beta_n(V) * n;
        double act = 1.0 / (1.0 + exp(-sig * (V - theta)));
        di[4] = act * (1.0 - s) / tau_r - s / tau_d;
    }
}

static int rhs_dim_ok(int rhs_id, int dim, int n_params)
{
    switch (rhs_id) {
    case FFO_LINEAR: return dim >= 1 && dim <= 8 && n_params == dim * dim;
    case FFO_HARMONIC: return dim == 2 && n_params == 1;
    case FFO_WILSON_COWAN: return dim == 2 && n_params == 10;
    case FFO_LORENZ: return dim == 3 && n_params == 3;
    case FFO_HH3: return dim == 15 && n_params == 16;
    default: return 0;
    }
}

static void rhs_eval(int rhs_id, int dim, const double *x, const double *p, double *dx)
{
    switch (rhs_id) {
    case FFO_LINEAR: rhs_linear(dim, x, p, dx); break;
    case FFO_HARMONIC: rhs_harmonic(x, p, dx); break;
    case FFO_WILSON_COWAN: rhs_wilson_cowan(x, p, dx); break;
    case FFO_LORENZ: rhs_lorenz(x, p, dx); break;
    case FFO_HH3: rhs_hh3(x, p, dx); break;
    }
}

/* One evaluation of f(x, p), exposed so tests can check it directly.
 * Returns 0 on success, -1 for an unknown system or a wrong size. */
int ffo_rhs(int rhs_id, int dim, const double *x, const double *p, int n_params, double *dx)
{
    if (!rhs_dim_ok(rhs_id, dim, n_params)) return -1;
    rhs_eval(rhs_id, dim, x, p, dx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Time steppers.                                                             */
/* ------------------------------------------------------------------------ */

/* Classical RK4 with constant step h (negative h integrates backward in
 * time):  k1 = f(x), k2 = f(x + h/2 k1), k3 = f(x + h/2 k2), k4 = f(x + h k3),
 *         x <- x + h/6 (k1 + 2 k2 + 2 k3 + k4). */
static void rk4_step(int rhs_id, int dim, double *x, const double *p, double h)
{
    double k1[FFO_MAXD], k2[FFO_MAXD], k3[FFO_MAXD], k4[FFO_MAXD], xs[FFO_MAXD];
    rhs_eval(rhs_id, dim, x, p, k1);
    for (int i = 0; i < dim; ++i) xs[i] = x[i] + (h / 2.0) * k1[i];
    rhs_eval(rhs_id, dim, xs, p, k2);
    for (int i = 0; i < dim; ++i) xs[i] = x[i] + (h / 2.0) * k2[i];
    rhs_eval(rhs_id, dim, xs, p, k3);
    for (int i = 0; i < dim; ++i) xs[i] = x[i] + h * k3[i];
    rhs_eval(rhs_id, dim, xs, p, k4);
    for (int i = 0; i < dim; ++i)
        x[i] = x[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Explicit Euler: x <- x + h f(x). */
static void euler_step(int rhs_id, int dim, double *x, const double *p, double h)
{
    double k[FFO_MAXD];
    rhs_eval(rhs_id, dim, x, p, k);
    for (int i = 0; i < dim; ++i) x[i] = x[i] + h * k[i];
}

/* Integrate P independent trajectories for n_steps constant steps.
 * state: SoA doubles, state[k * pitch + i].  h[i]: the step of particle i
 * (its group's direction times dt).  If pparam_index >= 0, parameter
 * pparam_index of particle i is pparam[i] instead of params[pparam_index].
 * Returns 0, or -1 on a bad argument. */
int ffo_integrate(int rhs_id, int method, int dim, int64_t P, int64_t pitch,
                  double *state, const double *params, int n_params,
                  int pparam_index, const double *pparam, const double *h,
                  int64_t n_steps)
{
    if (!rhs_dim_ok(rhs_id, dim, n_params)) return -1;
    if (method != FFO_RK4 && method != FFO_EULER) return -1;
    if (pparam_index >= n_params || (pparam_index >= 0 && !pparam)) return -1;
    if (pitch < P || n_steps < 0) return -1;
    double p[64];
    if (n_params > 64) return -1;
    for (int64_t i = 0; i < P; ++i) {
        double x[FFO_MAXD];
        for (int k = 0; k < dim; ++k) x[k] = state[(int64_t)k * pitch + i];
        memcpy(p, params, sizeof(double) * (size_t)n_params);
        if (pparam_index >= 0) p[pparam_index] = pparam[i];
        for (int64_t s = 0; s < n_steps; ++s) {
            if (method == FFO_RK4) rk4_step(rhs_id, dim, x, p, h[i]);
            else euler_step(rhs_id, dim, x, p, h[i]);
        }
        for (int k = 0; k < dim; ++k) state[(int64_t)k * pitch + i] = x[k];
    }
    return 0;
}

/* Integration with the paper's particle reset (Sec. 2.1: trajectories that
 * leave the box of valid states, or that have not been reset for more than
 * T_max, get new random initial conditions; Appendix A: state-variable bounds,
 * group initial-condition boxes).  The paper resets on the CPU, a batch per
 * frame; here the rule is applied every check_every steps:
 *   after each step the particle's age grows by one step; at global step
 *   numbers (step0 + s + 1) that are multiples of check_every, a particle whose
 *   state, rounded to float (the state array's precision), lies outside
 *   [blo_k, bhi_k] for some k (or is not finite), or whose age has reached
 *   max_age steps (max_age > 0), is re-drawn from its group's box: its r-th
 *   reset (r = resets + 1) uses draws n = (r * count + j) * dim + k + 1 of the
 *   group's SplitMix64 stream (j its index in the group, count the group's
 *   size), i.e. the blocks after the one used for its initial conditions;
 *   then age = 0 and resets = r.
 * blo/bhi may be NULL (no bounds).  Per particle: j[i], count[i], seed[i],
 * box lo/hi in lo[k * P + i], hi[k * P + i].  age/resets are updated in place.
 * Returns 0, or -1 on a bad argument. */
int ffo_integrate_reset(int rhs_id, int method, int dim, int64_t P, double *state,
                        const double *params, int n_params, int pparam_index, const double *pparam,
                        const double *h, int64_t n_steps, int64_t step0, int check_every,
                        const float *blo, const float *bhi, uint32_t max_age,
                        const int64_t *j, const int64_t *count, const uint64_t *seed,
                        const double *lo, const double *hi, uint32_t *age, uint32_t *resets)
{
    if (!rhs_dim_ok(rhs_id, dim, n_params)) return -1;
    if (method != FFO_RK4 && method != FFO_EULER) return -1;
    if (pparam_index >= n_params || (pparam_index >= 0 && !pparam)) return -1;
    if (n_steps < 0 || check_every < 1 || step0 < 0) return -1;
    if (n_params > 64) return -1;
    double p[64];
    for (int64_t i = 0; i < P; ++i) {
        double x[FFO_MAXD];
        for (int k = 0; k < dim; ++k) x[k] = state[(int64_t)k * P + i];
        memcpy(p, params, sizeof(double) * (size_t)n_params);
        if (pparam_index >= 0) p[pparam_index] = pparam[i];
        for (int64_t s = 0; s < n_steps; ++s) {
            if (method == FFO_RK4) rk4_step(rhs_id, dim, x, p, h[i]);
            else euler_step(rhs_id, dim, x, p, h[i]);
            age[i] += 1u;
            if ((step0 + s + 1) % check_every != 0) continue;
            int out = 0;
            if (blo && bhi) {
                for (int k = 0; k < dim; ++k) {
                    float xf = (float)x[k];
                    if (!(xf >= blo[k] && xf <= bhi[k])) out = 1;
                }
            }
            if (max_age > 0 && age[i] >= max_age) out = 1;
            if (!out) continue;
            uint32_t r = resets[i] + 1u;
            for (int k = 0; k < dim; ++k) {
                uint64_t n = ((uint64_t)r * (uint64_t)count[i] + (uint64_t)j[i]) * (uint64_t)dim + (uint64_t)k + 1u;
                uint64_t z = ffo_splitmix64(seed[i], n);
                double u = (double)(z >> 40) * (1.0 / 16777216.0);
                double width = hi[(int64_t)k * P + i] - lo[(int64_t)k * P + i];
                x[k] = (double)(float)(lo[(int64_t)k * P + i] + width * u);
            }
            age[i] = 0u;
            resets[i] = r;
        }
        for (int k = 0; k < dim; ++k) state[(int64_t)k * P + i] = x[k];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Derivatives for gradient checks (the paper has no gradients; these serve  */
/* the adjoint of the integrator).                                           */
/* ------------------------------------------------------------------------ */

/* Jacobian J[i*dim + k] = d f_i / d x_k and parameter Jacobian
 * Fp[i*n_params + q] = d f_i / d p_q, differentiated by hand from the right-hand
 * sides above.  Returns 0, or -1 for a system without derivatives here. */
static int rhs_jacobians(int rhs_id, int dim, const double *x, const double *p, int n_params,
                         double *J, double *Fp)
{
    for (int i = 0; i < dim * dim; ++i) J[i] = 0.0;
    for (int i = 0; i < dim * n_params; ++i) Fp[i] = 0.0;
    switch (rhs_id) {
    case FFO_LINEAR:
        for (int i = 0; i < dim; ++i) {
            for (int k = 0; k < dim; ++k) J[i * dim + k] = p[i * dim + k];
            for (int k = 0; k < dim; ++k) Fp[i * n_params + i * dim + k] = x[k];  /* d(Ax)_i / dA_ik */
        }
        return 0;
    case FFO_HARMONIC: {
        double w = p[0];
        J[0 * 2 + 1] = 1.0;
        J[1 * 2 + 0] = -(w * w);
        Fp[1 * n_params + 0] = -2.0 * w * x[0];
        return 0;
    }
    case FFO_LORENZ: {
        double sigma = p[0], r = p[1], beta = p[2];
        J[0] = -sigma; J[1] = sigma; J[2] = 0.0;
        J[3] = r - x[2]; J[4] = -1.0; J[5] = -x[0];
        J[6] = x[1]; J[7] = x[0]; J[8] = -beta;
        Fp[0 * 3 + 0] = x[1] - x[0];
        Fp[1 * 3 + 1] = x[0];
        Fp[2 * 3 + 2] = -x[2];
        return 0;
    }
    case FFO_WILSON_COWAN: {
        double E = x[0], I = x[1];
        double wEE = p[0], wEI = p[1], wIE = p[2], wII = p[3];
        double P = p[4], Q = p[5], tauE = p[6], tauI = p[7], gain = p[8], th = p[9];
        double aE = wEE * E - wEI * I + P, aI = wIE * E - wII * I + Q;
        double SE = wc_sigmoid(aE, gain, th), SI = wc_sigmoid(aI, gain, th);
        double dSE = gain * SE * (1.0 - SE), dSI = gain * SI * (1.0 - SI);  /* S'(a) */
        double fE = (-E + SE) / tauE, fI = (-I + SI) / tauI;
        J[0] = (-1.0 + dSE * wEE) / tauE;
        J[1] = (-dSE * wEI) / tauE;
        J[2] = (dSI * wIE) / tauI;
        J[3] = (-1.0 - dSI * wII) / tauI;
        /* dS/dgain = S (1 - S) (a - th), dS/dth = -gain S (1 - S) */
        Fp[0 * 10 + 0] = dSE * E / tauE;
        Fp[0 * 10 + 1] = -dSE * I / tauE;
        Fp[0 * 10 + 4] = dSE / tauE;
        Fp[0 * 10 + 6] = -fE / tauE;
        Fp[0 * 10 + 8] = SE * (1.0 - SE) * (aE - th) / tauE;
        Fp[0 * 10 + 9] = -dSE / tauE;
        Fp[1 * 10 + 2] = dSI * E / tauI;
        Fp[1 * 10 + 3] = -dSI * I / tauI;
        Fp[1 * 10 + 5] = dSI / tauI;
        Fp[1 * 10 + 7] = -fI / tauI;
        Fp[1 * 10 + 8] = SI * (1.0 - SI) * (aI - th) / tauI;
        Fp[1 * 10 + 9] = -dSI / tauI;
        return 0;
    }
    case FFO_HH3: {
        /* Eq. 6-11 differentiated term by term.  Gate rates depend on V only;
         * the rate constants are fixed numbers, not parameters. */
        double C = p[0], gNa = p[1], gK = p[2], gL = p[3];
        double ENa = p[4], EK = p[5], EL = p[6], gsyn = p[7], Esyn = p[8];
        double tau_r = p[12], tau_d = p[13], sig = p[14], theta = p[15];
        const int np = n_params;
        for (int i = 0; i < 3; ++i) {
            const double *xi = x + 5 * i;
            double V = xi[0], m = xi[1], h = xi[2], n = xi[3], s = xi[4];
            double s_others = 0.0;
            for (int j = 0; j < 3; ++j)
                if (j != i) s_others += x[5 * j + 4];
            double m3h = m * m * m * h, n4 = n * n * n * n;
            double Itot = gL * (EL - V) + gNa * m3h * (ENa - V) + gK * n4 * (EK - V) +
                          gsyn * (Esyn - V) * s_others + p[9 + i];
            int rV = 5 * i, rm = rV + 1, rh = rV + 2, rn = rV + 3, rs = rV + 4;
            /* voltage row */
            J[rV * dim + rV] = (-gL - gNa * m3h - gK * n4 - gsyn * s_others) / C;
            J[rV * dim + rm] = 3.0 * gNa * m * m * h * (ENa - V) / C;
            J[rV * dim + rh] = gNa * m * m * m * (ENa - V) / C;
            J[rV * dim + rn] = 4.0 * gK * n * n * n * (EK - V) / C;
            for (int j = 0; j < 3; ++j)
                if (j != i) J[rV * dim + 5 * j + 4] = gsyn * (Esyn - V) / C;
            Fp[rV * np + 0] = -Itot / (C * C);
            Fp[rV * np + 1] = m3h * (ENa - V) / C;
            Fp[rV * np + 2] = n4 * (EK - V) / C;
            Fp[rV * np + 3] = (EL - V) / C;
            Fp[rV * np + 4] = gNa * m3h / C;
            Fp[rV * np + 5] = gK * n4 / C;
            Fp[rV * np + 6] = gL / C;
            Fp[rV * np + 7] = (Esyn - V) * s_others / C;
            Fp[rV * np + 8] = gsyn * s_others / C;
            Fp[rV * np + 9 + i] = 1.0 / C;
            /* gates: d/dV of a(V)(1 - y) - b(V) y, and -(a + b) on the diagonal */
            double am = hh_alpha_m(V), bm = hh_beta_m(V), ah = hh_alpha_h(V), bh = hh_beta_h(V);
            double an = hh_alpha_n(V), bn = hh_beta_n(V);
            double dam = 0.1 * hh_vtrap_deriv(V + 40.0), dbm = -bm / 18.0;
            double dah = -ah / 20.0, dbh = bh * (1.0 - bh) / 10.0;
            double dan = 0.01 * hh_vtrap_deriv(V + 55.0), dbn = -bn / 80.0;
            J[rm * dim + rV] = dam * (1.0 - m) - dbm * m;
            J[rm * dim + rm] = -(am + bm);
            J[rh * dim + rV] = dah * (1.0 - h) - dbh * h;
            J[rh * dim + rh] = -(ah + bh);
            J[rn * dim + rV] = dan * (1.0 - n) - dbn * n;
            J[rn * dim + rn] = -(an + bn);
            /* synapse: act = 1 / (1 + exp(-sig (V - theta))), act' = sig act (1 - act) */
            double act = 1.0 / (1.0 + exp(-sig * (V - theta)));
            double a1 = act * (1.0 - act);
            J[rs * dim + rV] = sig * a1 * (1.0 - s) / tau_r;
            J[rs * dim + rs] = -act / tau_r - 1.0 / tau_d;
            Fp[rs * np + 12] = -act * (1.0 - s) / (tau_r * tau_r);
            Fp[rs * np + 13] = s / (tau_d * tau_d);
            Fp[rs * np + 14] = a1 * (V - theta) * (1.0 - s) / tau_r;
            Fp[rs * np + 15] = -sig * a1 * (1.0 - s) / tau_r;
        }
        return 0;
    }
    default:
        return -1;
    }
}

/* Jacobians exposed for tests. */
int ffo_jacobians(int rhs_id, int dim, const double *x, const double *p, int n_params, double *J, double *Fp)
{
    if (!rhs_dim_ok(rhs_id, dim, n_params)) return -1;
    return rhs_jacobians(rhs_id, dim, x, p, n_params, J, Fp);
}

#define FFO_AUG_MAX (16 + 16 * 16 + 16 * 64)

/* Right-hand side of the variational system y = (x, S, Q):
 *   dx/dt = f(x, p),  dS/dt = J(x) S,  dQ/dt = J(x) Q + F_p(x). */
static int aug_rhs(int rhs_id, int dim, int np, const double *y, const double *p, double *dy)
{
    double J[16 * 16], Fp[16 * 64];
    const double *x = y, *S = y + dim, *Q = y + dim + dim * dim;
    double *dx = dy, *dS = dy + dim, *dQ = dy + dim + dim * dim;
    if (rhs_jacobians(rhs_id, dim, x, p, np, J, Fp) != 0) return -1;
    rhs_eval(rhs_id, dim, x, p, dx);
    for (int i = 0; i < dim; ++i) {
        for (int c = 0; c < dim; ++c) {
            double s = 0.0;
            for (int k = 0; k < dim; ++k) s += J[i * dim + k] * S[k * dim + c];
            dS[i * dim + c] = s;
        }
        for (int q = 0; q < np; ++q) {
            double s = Fp[i * np + q];
            for (int k = 0; k < dim; ++k) s += J[i * dim + k] * Q[k * np + q];
            dQ[i * np + q] = s;
        }
    }
    return 0;
}

/* Forward sensitivities of the trajectories: the stepper (RK4 or Euler)
 * applied to the variational system, which gives exactly the derivatives of
 * the discrete map (the stages of the augmented system are the chain rule of the stages of
 * the original one).  Per particle i: xT[k*P+i], S[i][dim][dim] = d x(T) / d x0,
 * Q[i][dim][n_params] = d x(T) / d p (with pparam_index >= 0 that column is the
 * derivative with respect to the particle's own value).  Returns 0, or -1. */
int ffo_tangent(int rhs_id, int method, int dim, int64_t P, const double *x0, const double *params, int n_params,
                int pparam_index, const double *pparam, const double *h, int64_t n_steps,
                double *xT, double *S, double *Q)
{
    if (!rhs_dim_ok(rhs_id, dim, n_params) || dim > 16 || n_params > 64 || n_steps < 0) return -1;
    if (method != FFO_RK4 && method != FFO_EULER) return -1;
    if (pparam_index >= n_params || (pparam_index >= 0 && !pparam)) return -1;
    const int n = dim + dim * dim + dim * n_params;
    double y[FFO_AUG_MAX], k1[FFO_AUG_MAX], k2[FFO_AUG_MAX], k3[FFO_AUG_MAX], k4[FFO_AUG_MAX], ys[FFO_AUG_MAX];
    double p[64];
    for (int64_t i = 0; i < P; ++i) {
        memcpy(p, params, sizeof(double) * (size_t)n_params);
        if (pparam_index >= 0) p[pparam_index] = pparam[i];
        for (int a = 0; a < n; ++a) y[a] = 0.0;
        for (int k = 0; k < dim; ++k) {
            y[k] = x0[(int64_t)k * P + i];
            y[dim + k * dim + k] = 1.0;
        }
        double hh = h[i];
        for (int64_t s = 0; s < n_steps; ++s) {
            if (aug_rhs(rhs_id, dim, n_params, y, p, k1)) return -1;
            if (method == FFO_EULER) {  /* Euler on the variational system: the derivative of x + h f(x) */
                for (int a = 0; a < n; ++a) y[a] = y[a] + hh * k1[a];
                continue;
            }
            for (int a = 0; a < n; ++a) ys[a] = y[a] + (hh / 2.0) * k1[a];
            aug_rhs(rhs_id, dim, n_params, ys, p, k2);
            for (int a = 0; a < n; ++a) ys[a] = y[a] + (hh / 2.0) * k2[a];
            aug_rhs(rhs_id, dim, n_params, ys, p, k3);
            for (int a = 0; a < n; ++a) ys[a] = y[a] + hh * k3[a];
            aug_rhs(rhs_id, dim, n_params, ys, p, k4);
            for (int a = 0; a < n; ++a) y[a] = y[a] + (hh / 6.0) * (k1[a] + 2.0 * k2[a] + 2.0 * k3[a] + k4[a]);
        }
        for (int k = 0; k < dim; ++k) xT[(int64_t)k * P + i] = y[k];
        memcpy(S + i * dim * dim, y + dim, sizeof(double) * (size_t)(dim * dim));
        memcpy(Q + i * dim * n_params, y + dim + dim * dim, sizeof(double) * (size_t)(dim * n_params));
    }
    return 0;
}

/* Escaped particle: some component is not finite or exceeds 1e30 in
 * magnitude.  flags[i] (optional) receives 1 for escaped particles. */
int64_t ffo_count_escaped(int dim, int64_t P, int64_t pitch, const double *state, uint8_t *flags)
{
    int64_t n = 0;
    for (int64_t i = 0; i < P; ++i) {
        int esc = 0;
        for (int k = 0; k < dim; ++k) {
            double v = state[(int64_t)k * pitch + i];
            if (!(fabs(v) <= 1e30)) esc = 1;
        }
        if (flags) flags[i] = (uint8_t)esc;
        n += esc;
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Projection and splatting, in FP32 with each operation rounded separately.  */
/* ------------------------------------------------------------------------ */

/* Map one coordinate to a pixel index: floor((a - lo) * scale) where scale =
 * extent / (hi - lo) is formed in double and rounded to float.  Returns the
 * index as a float; the caller keeps it iff 0 <= index < extent. */
static float pixel_coord(float a, float lo_f, float scale_f)
{
    float d = a - lo_f;
    float q = d * scale_f;
    return floorf(q);
}

/* 2D render technique (Appendix A, vertex shader with a 2D camera): state
 * variables (u, v) map linearly to columns and rows of a W x H window showing
 * [lo_u, hi_u) x [lo_v, hi_v); row 0 is v = lo_v.  Each kept particle adds 1
 * to its pixel (fragment shader, additive blending), image[row * W + col].
 * include (optional) selects particles. */
void ffo_splat2d(int64_t P, const float *u, const float *v, const uint8_t *include,
                 double lo_u, double hi_u, double lo_v, double hi_v,
                 int W, int H, uint32_t *image)
{
    float lo_uf = (float)lo_u, lo_vf = (float)lo_v;
    float su = (float)((double)W / (hi_u - lo_u));
    float sv = (float)((double)H / (hi_v - lo_v));
    float Wf = (float)W, Hf = (float)H;
    for (int64_t i = 0; i < P; ++i) {
        if (include && !include[i]) continue;
        float c = pixel_coord(u[i], lo_uf, su);
        float r = pixel_coord(v[i], lo_vf, sv);
        if (c >= 0.0f && c < Wf && r >= 0.0f && r < Hf)
            image[(int64_t)r * W + (int64_t)c] += 1u;
    }
}

/* Soft-sprite render technique (Appendix A: the geometry shader emits a square
 * facing the camera and centred on the projected particle; the fragment shader
 * gives each pixel of that square an intensity that falls off smoothly with the
 * pixel's distance from the centre, giving a round particle; the blend
 * glBlendFunc(GL_SRC_ALPHA, GL_ONE) adds intensity times the particle's colour
 * to what the pixel already holds).  The paper gives neither the square's size
 * nor the falloff; the readings taken here:
 *  - the particle's centre, in continuous pixel units, is (a - lo) * scale on
 *    each axis: the count splat's coordinate before its floor;
 *  - pixel (col, row) is sampled at its centre (col + 1/2, row + 1/2); with the
 *    square's half-side R and q = (dx^2 + dy^2) / R^2 the pixel is covered iff
 *    q < 1 and gets intensity a = (1 - q)^2, which meets zero with zero slope at
 *    the rim (the square's corners, q >= 1, get nothing);
 *  - channel k (0..3) of the pixel gains gain * a * colour[g][k], g the
 *    particle's group; the image is [H][W][4] with the channels interleaved.
 * Coverage (q < 1) is decided in FP32 with every operation rounded on its own,
 * like the pixel rule; the intensities and sums are formed in double.
 * abs_image (optional) receives the sums of |contribution| per channel and
 * frags (optional) the number of fragments per pixel: the scale of the rounding
 * error of any FP32 summation of the same contributions. */
static void sprite_add(double *image, double *abs_image, uint32_t *frags, int W, int H,
                       float pc, float pr, float R, float inv_r2, double gain, const double *colour)
{
    /* the comparisons also reject non-finite centres */
    if (!(pc > -R - 1.0f && pc < (float)W + R + 1.0f && pr > -R - 1.0f && pr < (float)H + R + 1.0f))
        return;
    int c0 = (int)floorf(pc - R), c1 = (int)ceilf(pc + R);
    int r0 = (int)floorf(pr - R), r1 = (int)ceilf(pr + R);
    if (c0 < 0) c0 = 0;
    if (r0 < 0) r0 = 0;
    if (c1 > W - 1) c1 = W - 1;
    if (r1 > H - 1) r1 = H - 1;
    for (int row = r0; row <= r1; ++row) {
        for (int col = c0; col <= c1; ++col) {
            float dx = ((float)col + 0.5f) - pc;
            float dy = ((float)row + 0.5f) - pr;
            float dx2 = dx * dx;
            float dy2 = dy * dy;
            float d2 = dx2 + dy2;
            float q = d2 * inv_r2;
            if (!(q < 1.0f)) continue;
            double a = (1.0 - (double)q) * (1.0 - (double)q);
            int64_t at = ((int64_t)row * W + col) * 4;
            for (int k = 0; k < 4; ++k) {
                double c = gain * a * colour[k];
                image[at + k] += c;
                if (abs_image) abs_image[at + k] += fabs(c);
            }
            if (frags) frags[(int64_t)row * W + col] += 1u;
        }
    }
}

/* 2D soft sprites: the window map of ffo_splat2d, then sprite_add.  group[i] is
 * particle i's group; colour holds 4 channel weights per group; radius R > 0
 * pixels (1/R^2 is formed in double and rounded to float). */
void ffo_sprites2d(int64_t P, const float *u, const float *v, const int32_t *group, const uint8_t *include,
                   double lo_u, double hi_u, double lo_v, double hi_v, int W, int H,
                   float R, double gain, const double *colour,
                   double *image, double *abs_image, uint32_t *frags)
{
    float lo_uf = (float)lo_u, lo_vf = (float)lo_v;
    float su = (float)((double)W / (hi_u - lo_u));
    float sv = (float)((double)H / (hi_v - lo_v));
    float inv_r2 = (float)(1.0 / ((double)R * (double)R));
    for (int64_t i = 0; i < P; ++i) {
        if (include && !include[i]) continue;
        float du = u[i] - lo_uf;
        float pc = du * su;
        float dv = v[i] - lo_vf;
        float pr = dv * sv;
        sprite_add(image, abs_image, frags, W, H, pc, pr, R, inv_r2, gain, colour + 4 * group[i]);
    }
}

/* 3D soft sprites: the perspective map of ffo_splat3d (particles with clip
 * w <= 0 dropped), then sprite_add with a square of constant size on screen
 * (the geometry shader builds it after the projection). */
void ffo_sprites3d(int64_t P, const float *x, const float *y, const float *z, const int32_t *group,
                   const uint8_t *include, const float *m, int W, int H,
                   float R, double gain, const double *colour,
                   double *image, double *abs_image, uint32_t *frags)
{
    float su = (float)((double)W / 2.0), sv = (float)((double)H / 2.0);
    float inv_r2 = (float)(1.0 / ((double)R * (double)R));
    for (int64_t i = 0; i < P; ++i) {
        if (include && !include[i]) continue;
        float cl[4];
        for (int j = 0; j < 4; ++j) {
            float a = m[0 + j] * x[i];
            float b = m[4 + j] * y[i];
            float c = m[8 + j] * z[i];
            float s = a + b;
            s = s + c;
            s = s + m[12 + j];
            cl[j] = s;
        }
        if (!(cl[3] > 0.0f)) continue;
        float nx = cl[0] / cl[3];
        float ny = cl[1] / cl[3];
        float pc = (nx - -1.0f) * su;
        float pr = (ny - -1.0f) * sv;
        sprite_add(image, abs_image, frags, W, H, pc, pr, R, inv_r2, gain, colour + 4 * group[i]);
    }
}

/* 3D render technique (Appendix A, vertex + geometry shaders): clip = M [x,1]
 * with M the column-major 4x4 Model-View-Projection matrix (element (row j,
 * column c) at m[4c + j]), each row summed left to right; particles with
 * clip w <= 0 (behind the camera) are dropped; normalised device coordinates
 * clip.xy / w then map [-1, 1) onto the W x H window with the 2D rule. */
void ffo_splat3d(int64_t P, const float *x, const float *y, const float *z,
                 const uint8_t *include, const float *m, int W, int H, uint32_t *image)
{
    float su = (float)((double)W / 2.0), sv = (float)((double)H / 2.0);
    float Wf = (float)W, Hf = (float)H;
    for (int64_t i = 0; i < P; ++i) {
        if (include && !include[i]) continue;
        float cl[4];
        for (int j = 0; j < 4; ++j) {
            float a = m[0 + j] * x[i];
            float b = m[4 + j] * y[i];
            float c = m[8 + j] * z[i];
            float s = a + b;
            s = s + c;
            s = s + m[12 + j];
            cl[j] = s;
        }
        if (!(cl[3] > 0.0f)) continue;
        float nx = cl[0] / cl[3];
        float ny = cl[1] / cl[3];
        float c = pixel_coord(nx, -1.0f, su);
        float r = pixel_coord(ny, -1.0f, sv);
        if (c >= 0.0f && c < Wf && r >= 0.0f && r < Hf)
            image[(int64_t)r * W + (int64_t)c] += 1u;
    }
}
