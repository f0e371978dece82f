"""Pins of the oracle's time steppers (RK4, Euler, signed steps) against closed forms.

* One classical RK4 step on dx/dt = A x is exactly x <- T(hA) x with the
  degree-4 Taylor polynomial T(Z) = I + Z + Z^2/2 + Z^3/6 + Z^4/24, so n steps
  are a matrix power; a dropped stage, a wrong weight or a wrong stage point
  changes T and fails here.
* Euler is x <- (I + hA) x.
* The harmonic oscillator's per-step energy factor under RK4 is exactly
  |T(i w h)|^2 = 1 - (wh)^6/72 + (wh)^8/576.
* The global error against exp(At) x0 falls by 2^4 when h halves (order 4).
* A negative step (backward-time group) is the same map with h -> -h.
"""
import numpy as np
import pytest
import scipy.linalg

import oracle


def _taylor4(Z):
    I = np.eye(Z.shape[0])
    Z2 = Z @ Z
    Z3 = Z2 @ Z
    Z4 = Z3 @ Z
    return I + Z + Z2 / 2.0 + Z3 / 6.0 + Z4 / 24.0


def _stable_matrix(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return M - (np.abs(np.linalg.eigvals(M).real).max() + 0.5) * np.eye(n)


@pytest.mark.parametrize("n,h,steps", [(1, 0.1, 50), (3, 0.05, 37), (5, -0.02, 64), (8, 0.01, 10)])
def test_rk4_linear_is_matrix_power(n, h, steps):
    A = _stable_matrix(n, 7 + n)
    rng = np.random.default_rng(n)
    x0 = rng.standard_normal((n, 4))
    got = oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), h, steps)
    want = np.linalg.matrix_power(_taylor4(h * A), steps) @ x0
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("h,steps", [(0.1, 30), (-0.05, 17)])
def test_euler_linear_is_matrix_power(h, steps):
    A = _stable_matrix(4, 3)
    x0 = np.random.default_rng(1).standard_normal((4, 3))
    got = oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), h, steps, method=oracle.EULER)
    want = np.linalg.matrix_power(np.eye(4) + h * A, steps) @ x0
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("omega,h", [(1.0, 0.1), (2.5, 0.05), (0.7, 0.3)])
def test_harmonic_energy_factor(omega, h):
    n = 200
    x0 = np.array([[1.0, 0.3], [0.0, -2.0]])  # two particles (x, v)
    got = oracle.integrate(oracle.HARMONIC, x0, [omega], h, n)
    E0 = omega ** 2 * x0[0] ** 2 + x0[1] ** 2
    E = omega ** 2 * got[0] ** 2 + got[1] ** 2
    z = omega * h
    factor = 1.0 - z ** 6 / 72.0 + z ** 8 / 576.0
    np.testing.assert_allclose(E / E0, factor ** n, rtol=1e-12)


def test_rk4_fourth_order_convergence():
    A = np.array([[0.0, 1.0, 0.0], [-4.0, -0.3, 0.5], [0.2, 0.0, -1.0]])
    x0 = np.array([[1.0], [0.5], [-0.25]])
    T = 2.0
    exact = scipy.linalg.expm(A * T) @ x0
    errs = []
    for n in (40, 80, 160):
        got = oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), T / n, n)
        errs.append(np.abs(got - exact).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14.0 < r1 < 18.0 and 14.0 < r2 < 18.0, errs


def test_euler_first_order_convergence():
    A = np.array([[-1.0, 2.0], [-2.0, -1.0]])
    x0 = np.array([[1.0], [0.0]])
    exact = scipy.linalg.expm(A * 1.0) @ x0
    e1 = np.abs(oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), 1 / 400, 400,
                                 method=oracle.EULER) - exact).max()
    e2 = np.abs(oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), 1 / 800, 800,
                                 method=oracle.EULER) - exact).max()
    assert 1.8 < e1 / e2 < 2.2


def test_backward_group_then_forward_returns():
    # n steps with -h then n steps with +h: exactly T(hA)^n T(-hA)^n x0, which differs from x0
    # only by O(n h^5) because T(hA) T(-hA) = I + O(h^5).
    A = np.array([[0.0, 1.0], [-9.0, 0.0]])
    x0 = np.array([[1.0, -0.5], [0.2, 3.0]])
    h, n = 0.01, 300
    back = oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), -h, n)
    fwd = oracle.integrate(oracle.LINEAR, back, A.reshape(-1), h, n)
    want = np.linalg.matrix_power(_taylor4(h * A), n) @ np.linalg.matrix_power(_taylor4(-h * A), n) @ x0
    np.testing.assert_allclose(fwd, want, rtol=1e-11, atol=1e-12)
    assert np.abs(fwd - x0).max() < 1e-6


def test_per_particle_step_sign():
    # Two groups in one call: particle 0 forward, particle 1 backward.
    A = np.array([[0.0, 1.0], [-1.0, 0.0]])
    x0 = np.array([[1.0, 1.0], [0.0, 0.0]])
    h = np.array([0.05, -0.05])
    got = oracle.integrate(oracle.LINEAR, x0, A.reshape(-1), h, 40)
    want_f = np.linalg.matrix_power(_taylor4(0.05 * A), 40) @ x0[:, :1]
    want_b = np.linalg.matrix_power(_taylor4(-0.05 * A), 40) @ x0[:, 1:]
    np.testing.assert_allclose(got[:, :1], want_f, rtol=1e-12)
    np.testing.assert_allclose(got[:, 1:], want_b, rtol=1e-12)


def test_zero_steps_is_identity_and_bad_args_rejected():
    x0 = np.array([[1.5], [2.5], [3.5]])
    np.testing.assert_array_equal(oracle.integrate(oracle.LORENZ, x0, [10, 28, 8 / 3], 0.01, 0), x0)
    with pytest.raises(ValueError):
        oracle.integrate(oracle.LORENZ, x0, [10, 28], 0.01, 1)
    with pytest.raises(ValueError):
        oracle.integrate(oracle.HH3, x0, [0.0] * 16, 0.01, 1)


def test_escape_count():
    st = np.array([[0.0, np.nan, 1.0, 2e30, 5.0],
                   [0.0, 0.0, np.inf, 1.0, -1e30]])
    n, flags = oracle.count_escaped(st)
    assert n == 3
    assert flags.tolist() == [False, True, True, True, False]


def test_fp32_evaluation_is_the_same_map_in_single_precision():
    """oracle.integrate_fp32 (the FP32 yardstick of the GPU parity bar) computes the same
    RK4 map in float32: on dx/dt = A x it matches the matrix power T(hA)^n in float32 to
    a few float32 ulps per step (and is visibly not the FP64 result), and on Lorenz one
    step from an exactly representable state lands within a few float32 ulps of the
    FP64 step."""
    A = _stable_matrix(3, 21)
    x0 = np.random.default_rng(5).standard_normal((3, 64)).astype(np.float32)
    h, n = 0.01, 100
    got = oracle.integrate_fp32(oracle.LINEAR, x0, A.reshape(-1).astype(np.float32), h, n)
    assert got.dtype == np.float32
    A32 = A.astype(np.float32).astype(np.float64)
    want = np.linalg.matrix_power(_taylor4(np.float64(np.float32(h)) * A32), n) @ x0.astype(np.float64)
    scale = np.maximum(np.abs(want), 1.0)
    err = np.abs(got - want) / scale
    assert err.max() <= n * 8 * 2.0**-24
    assert err.max() > 1e-9  # rounded in FP32, not FP64
    x = np.array([[1.5], [-2.25], [20.0]], np.float32)
    p = [10.0, 28.0, 8.0 / 3.0]
    one32 = oracle.integrate_fp32(oracle.LORENZ, x, p, 0.001, 1).astype(np.float64)
    one64 = oracle.integrate(oracle.LORENZ, x, np.float32(p).astype(np.float64), np.float64(np.float32(0.001)), 1)
    assert np.all(np.abs(one32 - one64) <= 4 * np.spacing(np.abs(one64).astype(np.float32)).astype(np.float64))
    assert not np.array_equal(one32, one64)
