"""Pins of the oracle's three-neuron Hodgkin-Huxley right-hand side (Eq. 6-11).

* Gate kinetics: at the textbook resting potential -65 mV the textbook steady
  gates m, h, n make dm/dt, dh/dt, dn/dt vanish (to their 4 printed digits), and the
  membrane current balances there (rest at -65 mV).
* The removable singularities of alpha_m (V = -40) and alpha_n (V = -55) are
  continuous, with limits 1 and 0.1, and v / (1 - exp(-v/10)) matches a 40-digit
  evaluation to rounding on both sides of them.
* Synapse (Eq. 11): far below threshold ds/dt = -s/tau_d, far above
  (1-s)/tau_r - s/tau_d, at threshold half the rise term.
* All-to-all coupling (Eq. 10): neuron i receives sum_{j != i} s_j, never its own s.
* Bifurcation facts printed in Sec. 3 for one neuron: repetitive firing exists past
  I ~ 6.25 and not below it; at I = 10 the resting fixed point is weakly unstable.
"""
import numpy as np
import pytest

import oracle
from conftest import load_golden
from paper_1505_00344_gb300.workloads import HH3_BASE

G = load_golden("hh_textbook.txt")


def params(I=(0.0, 0.0, 0.0), gsyn=0.0):
    p = list(HH3_BASE)
    p[7] = gsyn
    p[9:12] = list(I)
    return p


def state(V, m, h, n, s):
    x = []
    for i in range(3):
        x += [V[i], m[i], h[i], n[i], s[i]]
    return np.array(x, dtype=np.float64)


def f(x, p):
    return oracle.rhs(oracle.HH3, x, p)


def test_resting_gates_textbook():
    V = float(G["V_rest"][0])
    m, h, n = float(G["m_inf"][0]), float(G["h_inf"][0]), float(G["n_inf"][0])
    x = state([V] * 3, [m] * 3, [h] * 3, [n] * 3, [0.0] * 3)
    d = f(x, params())
    for i in range(3):
        # derivative of each gate relative to its rate scale: 4-digit table -> ~1e-3
        assert abs(d[5 * i + 1]) < 4.3 * 6e-5 * 1.5
        assert abs(d[5 * i + 2]) < 0.12 * 6e-5 * 1.5
        assert abs(d[5 * i + 3]) < 0.19 * 6e-5 * 1.5
        assert abs(d[5 * i + 0]) < 0.05  # currents balance at rest (uA/cm^2 per uF/cm^2)


def test_resting_potential_reached():
    x0 = state([-70.0, -60.0, -65.0], [0.1, 0.0, 0.05], [0.5, 0.7, 0.6], [0.3, 0.35, 0.32], [0, 0, 0])
    x = oracle.integrate(oracle.HH3, x0.reshape(15, 1), params(), 0.01, 20000)
    for i in range(3):
        assert abs(x[5 * i, 0] - float(G["V_rest"][0])) < 0.05
        assert abs(x[5 * i + 1, 0] - float(G["m_inf"][0])) < 2e-4
        assert abs(x[5 * i + 2, 0] - float(G["h_inf"][0])) < 2e-4
        assert abs(x[5 * i + 3, 0] - float(G["n_inf"][0])) < 2e-4


@pytest.mark.parametrize("Vs,limit_alpha", [(-40.0, 1.0), (-55.0, 0.1)])
def test_removable_singularities(Vs, limit_alpha):
    # alpha(V) = dm/dt at m = 0 (for -40) / dn/dt at n = 0 (for -55) since (1-gate) = 1.
    gate = 1 if Vs == -40.0 else 3
    vals = []
    for dv in (-2e-4, -1.0001e-4, -0.9999e-4, 0.0, 0.9999e-4, 1.0001e-4, 2e-4):
        x = state([Vs + dv] * 3, [0.0] * 3, [0.0] * 3, [0.0] * 3, [0.0] * 3)
        vals.append(f(x, params())[gate])
    vals = np.array(vals)
    assert abs(vals[3] - limit_alpha) < 1e-12
    assert np.abs(np.diff(vals)).max() < 1e-5 * limit_alpha


def test_vtrap_series_high_precision():
    # alpha_m(V)/0.1 = v / (1 - exp(-v/10)) with v = V + 40; compare the oracle against a
    # 40-digit evaluation near and away from the removable singularity.
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for v in (3e-9, 3e-5, -7e-5, 9.9e-5, 2e-4, -0.3, 1.7, 25.0):
        x = state([-40.0 + v] * 3, [0.0] * 3, [0.0] * 3, [0.0] * 3, [0.0] * 3)
        # dm/dt at m = 0 is alpha_m; -40 + v rounds v to a multiple of ulp(40) ~ 7e-15
        vv = (-40.0 + v) + 40.0
        want = float(mpmath.mpf(vv) / (1 - mpmath.exp(-mpmath.mpf(vv) / 10)))
        got = f(x, params())[1] / 0.1
        assert abs(got - want) <= 2e-14 * abs(want)


def test_synapse_equation():
    p = params()
    tau_r, tau_d, theta = p[12], p[13], p[15]
    for s in (0.0, 0.3, 1.0):
        lo = f(state([-200.0] * 3, [0] * 3, [0] * 3, [0] * 3, [s] * 3), p)[4]
        hi = f(state([200.0] * 3, [0] * 3, [0] * 3, [0] * 3, [s] * 3), p)[4]
        mid = f(state([theta] * 3, [0] * 3, [0] * 3, [0] * 3, [s] * 3), p)[4]
        assert abs(lo + s / tau_d) < 1e-12
        assert abs(hi - ((1 - s) / tau_r - s / tau_d)) < 1e-12
        assert abs(mid - (0.5 * (1 - s) / tau_r - s / tau_d)) < 1e-12


def test_all_to_all_coupling_targets():
    p = params(gsyn=0.5)
    V = [-60.0, -60.0, -60.0]
    base = f(state(V, [0.05] * 3, [0.6] * 3, [0.3] * 3, [0, 0, 0]), p)
    one = f(state(V, [0.05] * 3, [0.6] * 3, [0.3] * 3, [0, 1.0, 0]), p)
    two = f(state(V, [0.05] * 3, [0.6] * 3, [0.3] * 3, [1.0, 1.0, 0]), p)
    unit = 0.5 * (-80.0 - (-60.0))  # gsyn (Esyn - V), inhibitory (negative)
    dv = lambda d: np.array([d[0], d[5], d[10]])
    np.testing.assert_allclose(dv(one) - dv(base), [unit, 0.0, unit], atol=1e-12)
    np.testing.assert_allclose(dv(two) - dv(base), [unit, unit, 2 * unit], atol=1e-12)


def test_drive_current_enters_own_neuron():
    a = f(state([-65.0] * 3, [0.05] * 3, [0.6] * 3, [0.32] * 3, [0] * 3), params(I=(0, 0, 0)))
    b = f(state([-65.0] * 3, [0.05] * 3, [0.6] * 3, [0.32] * 3, [0] * 3), params(I=(1.0, 2.0, 3.0)))
    np.testing.assert_allclose([b[0] - a[0], b[5] - a[5], b[10] - a[10]], [1.0, 2.0, 3.0],
                               atol=1e-12)


def _spikes(I, x0, t_ms, tail_ms, dt=0.01):
    """Integrate three uncoupled neurons with drive I; count upward V=0 crossings of neuron 1
    during the last tail_ms."""
    p = params(I=(I, I, I))
    x = x0.reshape(15, 1).copy()
    n_pre = int((t_ms - tail_ms) / dt)
    x = oracle.integrate(oracle.HH3, x, p, dt, n_pre)
    spikes, prev = 0, x[0, 0]
    chunk = 10
    for _ in range(int(tail_ms / dt) // chunk):
        x = oracle.integrate(oracle.HH3, x, p, dt, chunk)
        if prev < 0.0 <= x[0, 0]:
            spikes += 1
        prev = x[0, 0]
    return spikes, x


def test_repetitive_firing_onset_near_paper_value():
    # Continuation down in I from a state on the I = 10 limit cycle: the cycle survives down to
    # just above the paper's onset value and is gone just below it.
    onset = float(G["firing_onset_I"][0])
    rest = state([-65.0] * 3, [0.0529] * 3, [0.5961] * 3, [0.3177] * 3, [0] * 3)
    _, x = _spikes(10.0, rest + np.array([20.0, 0, 0, 0, 0] * 3), 100.0, 10.0)
    for I in (9.0, 8.0, 7.0):
        _, x = _spikes(I, x[:, 0], 100.0, 10.0)
    above, x = _spikes(onset + 0.25, x[:, 0], 150.0, 100.0)
    below, _ = _spikes(onset - 0.25, x[:, 0], 150.0, 100.0)
    assert above >= 3 and below == 0


def _rest_jacobian(I):
    p = params(I=(I, I, I))
    x = state([-65.0] * 3, [0.05] * 3, [0.6] * 3, [0.32] * 3, [0] * 3)
    for _ in range(50):  # Newton on the decoupled neuron 1 (4 variables)
        J = np.empty((15, 15))
        for j in range(15):
            e = np.zeros(15); e[j] = 1e-6
            J[:, j] = (f(x + e, p) - f(x - e, p)) / 2e-6
        d = f(x, p)
        x = x - np.linalg.solve(J + 1e-12 * np.eye(15), d)
    sub = [0, 1, 2, 3]
    return J[np.ix_(sub, sub)], np.abs(f(x, p)).max()


def test_rest_weakly_unstable_at_paper_drive():
    I_paper = float(G["weakly_unstable_I"][0])
    J, res = _rest_jacobian(I_paper)
    assert res < 1e-9
    lead = np.linalg.eigvals(J).real.max()
    assert 0.0 < lead < 0.05  # unstable, but only weakly (per ms)
    J8, _ = _rest_jacobian(8.0)
    assert np.linalg.eigvals(J8).real.max() < 0.0
