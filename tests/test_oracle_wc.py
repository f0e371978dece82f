"""Pins of the oracle's Wilson-Cowan right-hand side (Eq. 1-2) and RK4 on it.

The logistic response S(a) = 1/(1+exp(-gain (a - threshold))) is pinned by its
special values (S(threshold) = 1/2, the symmetry S(th+d) + S(th-d) = 1, slope
gain/4 at the threshold, saturation to 0 and 1).  Each coupling weight is pinned
by its sign and by the population it enters.  With all weights zero the system is
linear with a constant drive, and RK4 is then exactly
E_n = S* + (E_0 - S*) T(-h/tau)^n with T the RK4 stability polynomial.  At the
workload's parameters the one equilibrium (Newton on Eq. 1-2) is a stable focus, and
the oracle's trajectories from the unit square spiral into it at its eigenvalues' rate.
"""
import math

import numpy as np
import pytest

import oracle

# [wEE, wEI, wIE, wII, P, Q, tauE, tauI, gain, threshold]
ZERO_W = [0.0, 0.0, 0.0, 0.0, 4.0, 4.0, 1.0, 1.0, 1.0, 4.0]


def f(E, I, p):
    return oracle.rhs(oracle.WILSON_COWAN, [E, I], p)


def sig_at(drive, gain=1.0, th=4.0):
    """Value of S(drive) as seen through dE/dt at E = I = 0 with weights 0."""
    p = [0.0, 0.0, 0.0, 0.0, drive, 0.0, 1.0, 1.0, gain, th]
    return f(0.0, 0.0, p)[0]


def test_sigmoid_special_values():
    assert sig_at(4.0) == 0.5
    assert sig_at(7.0, gain=3.0, th=7.0) == 0.5
    for d in (0.3, 1.0, 5.0):
        assert abs(sig_at(4.0 + d) + sig_at(4.0 - d) - 1.0) < 1e-15
    assert sig_at(5.0) > 0.5 > sig_at(3.0)  # increasing
    for gain in (1.0, 2.0, 0.25):
        eps = 1e-6
        slope = (sig_at(4.0 + eps, gain) - sig_at(4.0 - eps, gain)) / (2 * eps)
        assert abs(slope - gain / 4.0) < 1e-8
    assert sig_at(4.0 + 60.0) >= 1 - 1e-15 and sig_at(4.0 - 60.0) < 1e-20


def test_coupling_signs_and_targets():
    base = list(ZERO_W)  # S(drive) = 1/2 for both populations when weights vanish
    # wEE excites E: dE at (E=1, I=0) = -1 + S(4 + wEE)
    p = list(base); p[0] = 2.0
    dE, dI = f(1.0, 0.0, p)
    assert dE > -0.5 and dI == 0.5
    # wEI inhibits E through I: dE at (E=0, I=1) = S(4 - wEI) < 1/2, dI untouched
    p = list(base); p[1] = 2.0
    dE, dI = f(0.0, 1.0, p)
    assert dE < 0.5 and dI == -1.0 + 0.5
    # wIE excites I through E: dI at (E=1, I=0) = S(4 + wIE) > 1/2 ... minus I = 0
    p = list(base); p[2] = 2.0
    dE, dI = f(1.0, 0.0, p)
    assert dI > 0.5 and dE == -0.5
    # wII inhibits I: dI at (E=0, I=1) = -1 + S(4 - wII) < -1/2
    p = list(base); p[3] = 2.0
    dE, dI = f(0.0, 1.0, p)
    assert dI < -0.5 and dE == 0.5
    # symmetric values: a unit of wEE at E = 1 is the mirror of a unit of wEI at I = 1
    p1 = list(base); p1[0] = 1.5
    p2 = list(base); p2[1] = 1.5
    assert abs((f(1.0, 0.0, p1)[0] + 1.0) + f(0.0, 1.0, p2)[0] - 1.0) < 1e-15


def test_time_constants_scale_rates():
    p = [16.0, 12.0, 15.0, 3.0, 1.25, 0.0, 1.0, 1.0, 1.0, 4.0]
    q = list(p); q[6] = 2.0; q[7] = 0.5
    a = f(0.3, 0.6, p)
    b = f(0.3, 0.6, q)
    assert abs(b[0] - a[0] / 2.0) < 1e-15 and abs(b[1] - a[1] * 2.0) < 1e-15


@pytest.mark.parametrize("h,n,tauE,tauI", [(0.01, 1000, 1.0, 1.0), (-0.01, 300, 1.0, 1.0),
                                           (0.05, 200, 2.0, 0.5)])
def test_zero_weights_closed_form(h, n, tauE, tauI):
    p = list(ZERO_W); p[4] = 5.0; p[5] = 2.0; p[6] = tauE; p[7] = tauI
    SE = 1.0 / (1.0 + math.exp(-(5.0 - 4.0)))
    SI = 1.0 / (1.0 + math.exp(-(2.0 - 4.0)))
    x0 = np.array([[0.1, 0.9], [0.7, 0.2]])
    got = oracle.integrate(oracle.WILSON_COWAN, x0, p, h, n)

    def T(z):
        return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24

    want_E = SE + (x0[0] - SE) * T(-h / tauE) ** n
    want_I = SI + (x0[1] - SI) * T(-h / tauI) ** n
    np.testing.assert_allclose(got[0], want_E, rtol=1e-12)
    np.testing.assert_allclose(got[1], want_I, rtol=1e-12)


def test_unit_square_forward_invariant_backward_leaves():
    # Since 0 < S < 1, dE/dt >= 0 at E = 0 and <= 0 at E = 1 (same for I): forward
    # trajectories started in [0,1]^2 stay there; backward ones (the paper's pink groups)
    # are pushed out of it unless they sit on a repeller.
    p = [16.0, 12.0, 15.0, 3.0, 1.25, 0.0, 1.0, 1.0, 1.0, 4.0]
    x0 = oracle.seed_group(2, [0, 0], [1, 1], 42, count=256).astype(np.float64)
    fwd = oracle.integrate(oracle.WILSON_COWAN, x0, p, 0.01, 1000)
    assert fwd.min() >= 0.0 and fwd.max() <= 1.0
    bwd = oracle.integrate(oracle.WILSON_COWAN, x0, p, -0.01, 1000)
    outside = (bwd < 0.0).any(axis=0) | (bwd > 1.0).any(axis=0)
    assert outside.mean() > 0.9


def test_config_fixed_point_is_the_attractor():
    # The workload's parameters (wEE=16, wEI=12, wIE=15, wII=3, P=1.25, Q=0, tau=1, gain 1,
    # threshold 4).  Its equilibria are the zeros of Eq. 1-2, found here by Newton's method on
    # the equations as the paper states them (not through the oracle), from a grid of starts in
    # the unit square: there is exactly one, and the trace and determinant of its Jacobian make
    # it a stable focus.  The oracle's forward trajectories from the whole square must then
    # spiral into it, their distance shrinking at the rate of the eigenvalues' real part.
    p = [16.0, 12.0, 15.0, 3.0, 1.25, 0.0, 1.0, 1.0, 1.0, 4.0]
    wEE, wEI, wIE, wII, P, Q = p[:6]

    def S(a):
        return 1.0 / (1.0 + math.exp(-(a - 4.0)))

    def F(x):
        E, I = x
        return np.array([-E + S(wEE * E - wEI * I + P), -I + S(wIE * E - wII * I + Q)])

    def J(x):
        E, I = x
        sE = S(wEE * E - wEI * I + P)
        sI = S(wIE * E - wII * I + Q)
        dE, dI = sE * (1.0 - sE), sI * (1.0 - sI)
        return np.array([[-1.0 + dE * wEE, -dE * wEI], [dI * wIE, -1.0 - dI * wII]])

    roots = []
    for E0 in np.linspace(0.0, 1.0, 11):
        for I0 in np.linspace(0.0, 1.0, 11):
            x = np.array([E0, I0])
            for _ in range(60):
                dx = np.linalg.solve(J(x), -F(x))
                x = x + dx
                if np.abs(dx).max() < 1e-14:
                    break
            if np.abs(F(x)).max() < 1e-13 and not any(np.abs(x - r).max() < 1e-9 for r in roots):
                roots.append(x)
    assert len(roots) == 1
    xs = roots[0]
    M = J(xs)
    tr, det = np.trace(M), np.linalg.det(M)
    assert tr < 0 and det > 0 and tr * tr < 4 * det  # stable focus
    re = tr / 2.0  # real part of both eigenvalues

    x0 = oracle.seed_group(2, [0, 0], [1, 1], 17, count=256).astype(np.float64)
    x1 = oracle.integrate(oracle.WILSON_COWAN, x0, p, 0.01, 3000)  # t = 30
    x2 = oracle.integrate(oracle.WILSON_COWAN, x1, p, 0.01, 3000)  # t = 60
    d1 = np.abs(x1 - xs[:, None]).max()
    d2 = np.abs(x2 - xs[:, None]).max()
    assert d2 < 2e-3
    # near the focus the distance shrinks by exp(re * 30) per 30 time units (the rotation
    # makes the max-norm ratio wander by a bounded factor)
    ratio = d2 / d1
    assert 0.5 * math.exp(re * 30.0) < ratio < 2.0 * math.exp(re * 30.0), (ratio, math.exp(re * 30.0))
