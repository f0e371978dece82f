"""Pins of the oracle's derivatives, used to check the CUDA adjoint.

* The hand-derived Jacobians d f/d x and d f/d p match central differences of the
  (already pinned) right-hand sides.
* For dx/dt = A x the sensitivity d x(T)/d x0 of n RK4 steps is exactly the matrix
  power T(hA)^n, and d x(T)/d A matches central differences of that closed form.
* The MSE gradients from the forward sensitivities match central differences of
  the loss computed with the plain integrator (Lorenz, Wilson-Cowan), including a
  per-particle parameter.
"""
import numpy as np
import pytest

import oracle
from paper_1505_00344_gb300.workloads import HH3_BASE, LORENZ_PARAMS, WC_PARAMS


def hh_state(V1, V2, V3):
    # neuron i: (V_i, m, h, n, s) with distinct gate values per neuron
    g = [(0.05, 0.6, 0.32, 0.1), (0.3, 0.2, 0.55, 0.7), (0.9, 0.05, 0.8, 0.45)]
    return [v for V, gi in zip((V1, V2, V3), g) for v in (V, *gi)]


def fd_jac(rid, x, p, eps=1e-6):
    x = np.asarray(x, float)
    p = np.asarray(p, float)
    J = np.empty((x.size, x.size))
    Fp = np.empty((x.size, p.size))
    for k in range(x.size):
        e = np.zeros_like(x); e[k] = eps * max(1.0, abs(x[k]))
        J[:, k] = (oracle.rhs(rid, x + e, p) - oracle.rhs(rid, x - e, p)) / (2 * e[k])
    for q in range(p.size):
        e = np.zeros_like(p); e[q] = eps * max(1.0, abs(p[q]))
        Fp[:, q] = (oracle.rhs(rid, x, p + e) - oracle.rhs(rid, x, p - e)) / (2 * e[q])
    return J, Fp


@pytest.mark.parametrize("rid,x,p", [
    (oracle.LORENZ, [3.0, -7.0, 25.0], LORENZ_PARAMS),
    (oracle.LORENZ, [-12.0, 4.0, 1.0], [9.0, 150.0, 2.0]),
    (oracle.WILSON_COWAN, [0.3, 0.6], WC_PARAMS),
    (oracle.WILSON_COWAN, [0.9, 0.1], [3.0, 5.0, 2.0, 1.0, 0.5, -1.0, 1.5, 0.7, 2.0, 3.0]),
    (oracle.HARMONIC, [0.4, -1.2], [2.5]),
    (oracle.LINEAR, [1.0, -2.0, 0.5], list(np.arange(9) * 0.3 - 1.0)),
    (oracle.HH3, hh_state(-63.0, -20.0, 12.5), HH3_BASE),
    # V at the removable points of alpha_m (-40) and alpha_n (-55), and just beside them
    (oracle.HH3, hh_state(-40.0, -55.0, -40.03), HH3_BASE),
    (oracle.HH3, hh_state(-54.96, -39.5, -85.0), [1.3, 100.0, 30.0, 0.5, 55.0, -70.0, -50.0, 0.9, -75.0,
                                                   7.0, 11.0, 13.0, 0.3, 6.0, 0.8, -15.0]),
])
def test_jacobians_match_central_differences(rid, x, p):
    J, Fp = oracle.jacobians(rid, x, p)
    Jf, Ff = fd_jac(rid, x, p)
    # per row of f: central differences are good to ~1e-9 of the row's largest entry
    scale = np.maximum(1.0, np.maximum(np.abs(Jf).max(axis=1), np.abs(Ff).max(axis=1)))[:, None]
    assert (np.abs(J - Jf) / scale).max() <= 1e-7
    assert (np.abs(Fp - Ff) / scale).max() <= 1e-7


def taylor4(Z):
    I = np.eye(Z.shape[0])
    return I + Z + Z @ Z / 2 + Z @ Z @ Z / 6 + Z @ Z @ Z @ Z / 24


def test_euler_sensitivity_is_matrix_power():
    A = np.array([[-0.5, 1.0], [-1.0, -0.3]])
    x0 = np.array([[1.0], [0.3]])
    h, n = 0.05, 30
    _, S, _ = oracle.tangent(oracle.LINEAR, x0, A.reshape(-1), h, n, method=oracle.EULER)
    np.testing.assert_allclose(S[0], np.linalg.matrix_power(np.eye(2) + h * A, n), rtol=1e-13, atol=1e-15)
    # and the Euler loss gradient matches central differences
    target = np.array([[0.2], [-0.1]])
    L, dx0, dp = oracle.mse_gradients(oracle.LINEAR, x0, A.reshape(-1), h, n, target, method=oracle.EULER)
    for k in range(2):
        e = np.zeros_like(x0); e[k, 0] = 1e-6
        lp = ((oracle.integrate(oracle.LINEAR, x0 + e, A.reshape(-1), h, n, method=oracle.EULER) - target) ** 2).sum()
        lm = ((oracle.integrate(oracle.LINEAR, x0 - e, A.reshape(-1), h, n, method=oracle.EULER) - target) ** 2).sum()
        assert abs(dx0[k, 0] - (lp - lm) / 2e-6) <= 1e-7


def test_linear_sensitivity_is_matrix_power():
    A = np.array([[-0.5, 1.0, 0.2], [-1.0, -0.3, 0.0], [0.1, 0.4, -0.8]])
    x0 = np.array([[1.0, -0.5], [0.3, 2.0], [-1.2, 0.7]])
    h, n = 0.05, 40
    xT, S, Q = oracle.tangent(oracle.LINEAR, x0, A.reshape(-1), h, n)
    M = np.linalg.matrix_power(taylor4(h * A), n)
    for i in range(2):
        np.testing.assert_allclose(S[i], M, rtol=1e-12, atol=1e-14)
    # d x(T) / d A_ab by central differences of the closed form
    eps = 1e-6
    for a in range(3):
        for b in range(3):
            E = np.zeros_like(A); E[a, b] = eps
            d = (np.linalg.matrix_power(taylor4(h * (A + E)), n) @ x0
                 - np.linalg.matrix_power(taylor4(h * (A - E)), n) @ x0) / (2 * eps)
            np.testing.assert_allclose(Q[:, :, a * 3 + b].T, d, rtol=1e-6, atol=1e-9)


def loss(rid, x0, p, h, n, target, **kw):
    xT = oracle.integrate(rid, x0, p, h, n, **kw)
    return float(((xT - target) ** 2).sum() / x0.shape[1])


@pytest.mark.parametrize("rid,params,box,h,n", [
    (oracle.LORENZ, LORENZ_PARAMS, ([-20, -20, 0], [20, 20, 40]), 0.001, 300),
    (oracle.WILSON_COWAN, WC_PARAMS, ([0, 0], [1, 1]), 0.01, 200),
    (oracle.HH3, HH3_BASE, ([-80, 0, 0, 0, 0] * 3, [40, 1, 1, 1, 1] * 3), 0.01, 150),
])
def test_mse_gradients_match_finite_differences(rid, params, box, h, n):
    dim = len(box[0])
    x0 = oracle.seed_group(dim, box[0], box[1], 17, count=6).astype(np.float64)
    target = oracle.seed_group(dim, box[0], box[1], 18, count=6).astype(np.float64)
    # HH3 run backward in time is unstable (the gates leave [0, 1]): forward steps only
    hh = np.array([h, h, h, h, h, h]) if rid == oracle.HH3 else np.array([h, -h, h, h, -h, h])
    L, dx0, dp = oracle.mse_gradients(rid, x0, params, hh, n, target)
    assert abs(L - loss(rid, x0, params, hh, n, target)) <= 1e-12 * max(1.0, L)
    # central differences with a step relative to the coordinate; the bar adds their
    # rounding floor, ~ 50 ulp of the loss divided by the step
    eps = 1e-6
    floor = 50 * np.finfo(float).eps * max(1.0, L)
    for k in range(dim):
        for i in range(6):
            e = np.zeros_like(x0); e[k, i] = eps * max(1.0, abs(x0[k, i]))
            fd = (loss(rid, x0 + e, params, hh, n, target) - loss(rid, x0 - e, params, hh, n, target)) / (2 * e[k, i])
            assert abs(dx0[k, i] - fd) <= 1e-6 * max(1.0, abs(fd)) + floor / e[k, i]
    for q in range(len(params)):
        e = np.zeros(len(params)); e[q] = eps * max(1.0, abs(params[q]))
        fd = (loss(rid, x0, np.add(params, e), hh, n, target) - loss(rid, x0, np.subtract(params, e), hh, n, target)) \
            / (2 * e[q])
        assert abs(dp[q] - fd) <= 1e-6 * max(1.0, abs(fd)) + floor / e[q]


def test_per_particle_parameter_column():
    x0 = oracle.seed_group(3, [-20, -20, 0], [20, 20, 40], 5, count=4).astype(np.float64)
    target = np.zeros_like(x0)
    r = np.array([5.0, 15.0, 28.0, 60.0])
    _, S, Q = oracle.tangent(oracle.LORENZ, x0, LORENZ_PARAMS, 0.001, 200, pparam_index=1, pparam=r)
    eps = 1e-6
    for i in range(4):
        rp, rm = r.copy(), r.copy()
        rp[i] += eps
        rm[i] -= eps
        d = (oracle.integrate(oracle.LORENZ, x0, LORENZ_PARAMS, 0.001, 200, pparam_index=1, pparam=rp)
             - oracle.integrate(oracle.LORENZ, x0, LORENZ_PARAMS, 0.001, 200, pparam_index=1, pparam=rm)) / (2 * eps)
        np.testing.assert_allclose(Q[i, :, 1], d[:, i], rtol=1e-6, atol=1e-7)
