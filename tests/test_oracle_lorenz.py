"""Pins of the oracle's Lorenz right-hand side (Eq. 3-5) and of RK4 on it.

Checked against the textbook fixed points C+- = (+-sqrt(beta(r-1)), +-sqrt(beta(r-1)), r-1),
the constant divergence -(sigma+1+beta), the closed-form eigenvalues at the origin,
and the bifurcation values the paper prints in Sec. 2.2: the pitchfork at r = 1, the
homoclinic bifurcation at r ~ 13.926 and the loss of stability of the spirals at
r ~ 24.74.
"""
import math

import numpy as np
import pytest

import oracle
from conftest import load_golden

G = load_golden("paper_lorenz.txt")
SIGMA = float(G["sigma"][0])
BETA = float(G["beta"][0])


def f(x, r, beta=BETA):
    return oracle.rhs(oracle.LORENZ, x, [SIGMA, r, beta])


def jac(x, r, beta=BETA, eps=1e-6):
    x = np.asarray(x, dtype=np.float64)
    J = np.empty((3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = eps
        J[:, j] = (f(x + e, r, beta) - f(x - e, r, beta)) / (2 * eps)
    return J


def c_plus(r, beta=BETA):
    a = math.sqrt(beta * (r - 1.0))
    return np.array([a, a, r - 1.0])


@pytest.mark.parametrize("r", [0.5, 5.0, 13.0, 28.0, 99.0])
def test_fixed_points_are_zeros(r):
    assert np.abs(f([0.0, 0.0, 0.0], r)).max() == 0.0
    if r > 1:
        for s in (1, -1):
            c = c_plus(r) * np.array([s, s, 1])
            assert np.abs(f(c, r)).max() < 1e-12 * max(1.0, r)


def test_divergence_constant():
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = rng.uniform(-20, 20, 3)
        r = rng.uniform(0, 100)
        assert abs(np.trace(jac(x, r)) + (SIGMA + 1 + BETA)) < 1e-6


@pytest.mark.parametrize("r", [0.5, 28.0])
def test_origin_eigenvalues(r):
    ev = np.sort_complex(np.linalg.eigvals(jac([0.0, 0.0, 0.0], r)))
    disc = (SIGMA + 1) ** 2 - 4 * SIGMA * (1 - r)
    want = np.sort_complex(np.array([-BETA, (-(SIGMA + 1) + math.sqrt(disc)) / 2,
                                     (-(SIGMA + 1) - math.sqrt(disc)) / 2], dtype=complex))
    np.testing.assert_allclose(ev, want, atol=1e-6)


def _max_re_at_cplus(r, beta=BETA):
    return np.linalg.eigvals(jac(c_plus(r, beta), r, beta)).real.max()


def test_spirals_lose_stability_where_paper_says():
    # bisection on the sign of the leading real part at C+
    lo, hi = 20.0, 30.0
    assert _max_re_at_cplus(lo) < 0 < _max_re_at_cplus(hi)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if _max_re_at_cplus(mid) < 0:
            lo = mid
        else:
            hi = mid
    paper = float(G["spirals_unstable_r"][0])  # printed with two decimals
    assert abs(lo - paper) < 0.005
    # and at beta = 2 (the value the bifurcation workload switches to) the textbook closed form
    lo2, hi2 = 15.0, 30.0
    for _ in range(40):
        mid = 0.5 * (lo2 + hi2)
        if _max_re_at_cplus(mid, 2.0) < 0:
            lo2 = mid
        else:
            hi2 = mid
    assert abs(lo2 - SIGMA * (SIGMA + 2.0 + 3) / (SIGMA - 2.0 - 1)) < 1e-4


def test_pitchfork_at_r_one():
    # Paper Sec. 2.2: below r = 1 everything approaches the origin; above it the origin is a
    # saddle and particles settle on C+ or C- with z = r - 1.
    assert float(G["pitchfork_r"][0]) == 1.0
    x0 = oracle.seed_group(3, [-10, -30, 0], [10, 30, 50], 11, count=32)
    low = oracle.integrate(oracle.LORENZ, x0, [SIGMA, 0.5, BETA], 0.01, 4000)
    assert np.abs(low).max() < 1e-3
    high = oracle.integrate(oracle.LORENZ, x0, [SIGMA, 5.0, BETA], 0.01, 4000)
    np.testing.assert_allclose(high[2], 4.0, atol=1e-3)
    np.testing.assert_allclose(np.abs(high[0]), c_plus(5.0)[0], atol=1e-3)
    assert (high[0] > 0).any() and (high[0] < 0).any()


def _settles_on_plus(r):
    # leave the saddle along its outgoing separatrix on the x > 0 side
    x0 = np.array([[1e-7], [1e-7], [0.0]])
    x = oracle.integrate(oracle.LORENZ, x0, [SIGMA, r, BETA], 0.002, 40000)
    return x[0, 0] > 0


def test_homoclinic_crossover_where_paper_says():
    paper = float(G["homoclinic_r"][0])
    lo, hi = 12.5, 15.5
    assert _settles_on_plus(lo) and not _settles_on_plus(hi)
    for _ in range(12):
        mid = 0.5 * (lo + hi)
        if _settles_on_plus(mid):
            lo = mid
        else:
            hi = mid
    assert abs(0.5 * (lo + hi) - paper) < 0.01


def test_per_particle_r_bifurcation_branches():
    # Per-particle parameter path: r_i from a linspace; for 2 <= r <= 8 every particle ends on
    # z = r - 1 (C+- branch), for r < 1 on the origin.  The beta switch mid-run keeps z = r - 1.
    P = 64
    r = oracle.linspace_param(P, 0.0, 10.0).astype(np.float64)
    x0 = oracle.seed_group(3, [-20, -20, 0], [20, 20, 40], 3, count=P)
    x = oracle.integrate(oracle.LORENZ, x0, [SIGMA, 28.0, BETA], 0.005, 4000, pparam_index=1,
                         pparam=r)
    x = oracle.integrate(oracle.LORENZ, x, [SIGMA, 28.0, 2.0], 0.005, 4000, pparam_index=1,
                         pparam=r)
    big = (r >= 2.0) & (r <= 8.0)
    np.testing.assert_allclose(x[2, big], r[big] - 1.0, atol=1e-4)
    small = r < 0.9
    assert np.abs(x[:, small]).max() < 1e-3
    # per-particle parameter equals a scalar-parameter run with that value
    one = oracle.integrate(oracle.LORENZ, x0[:, 40:41], [SIGMA, float(r[40]), BETA], 0.005, 100)
    many = oracle.integrate(oracle.LORENZ, x0, [SIGMA, 28.0, BETA], 0.005, 100, pparam_index=1,
                            pparam=r)
    np.testing.assert_array_equal(one[:, 0], many[:, 40])


def test_chaotic_at_classical_r():
    # r = 28 is past the strange-attractor value the paper prints: a generic trajectory keeps
    # visiting both lobes instead of settling on a spiral.
    x0 = np.array([[1.0], [1.0], [1.0]])
    x = x0
    signs = set()
    for _ in range(40):
        x = oracle.integrate(oracle.LORENZ, x, [SIGMA, 28.0, BETA], 0.001, 500)
        signs.add(bool(x[0, 0] > 0))
    assert signs == {True, False}
    assert float(G["strange_attractor_r"][0]) < 28.0


def test_rk4_commutes_with_the_z_shift():
    """RK4 commutes with affine changes of variables, so stepping Lorenz in zt = z - r
    (where the right-hand side reads (sigma (y - x), -(x zt + y), x y - beta zt - beta r))
    is the same map: the FP64 oracle's steps and the shifted steps agree to rounding, for
    forward and backward steps.  The CUDA integrators step in zt."""
    rng = np.random.default_rng(11)
    r = 28.0
    x0 = np.stack([rng.uniform(-20, 20, 64), rng.uniform(-20, 20, 64), rng.uniform(0, 40, 64)])

    def fs(s):
        x, y, zt = s
        return np.stack([SIGMA * (y - x), -(x * zt + y), x * y - BETA * zt - BETA * r])

    for h in (0.001, -0.001):
        want = oracle.integrate(oracle.LORENZ, x0.copy(), [SIGMA, r, BETA], np.full(64, h), 200)
        s = x0 - np.array([[0.0], [0.0], [r]])
        for _ in range(200):
            k1 = fs(s)
            k2 = fs(s + 0.5 * h * k1)
            k3 = fs(s + 0.5 * h * k2)
            k4 = fs(s + h * k3)
            s = s + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        got = s + np.array([[0.0], [0.0], [r]])
        assert np.abs(got - want).max() <= 1e-10 * max(1.0, np.abs(want).max())
