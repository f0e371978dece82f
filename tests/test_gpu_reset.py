"""GPU parity of the in-kernel particle reset (Sec. 2.1, Appendix A) against the oracle.

* Age-limit resets are integer decisions: ages and reset counts are exact, and the
  re-drawn initial conditions are the oracle's draws bit for bit, so states agree to
  the usual integration tolerance over the steps since the last reset.
* Bounds resets compare the float state with the bounds on both sides; a particle
  within rounding of a bound at a check step may decide differently in FP32 and
  FP64, so at least 99% of particles must agree on (age, resets) and those must
  agree in state.
* The check schedule follows global step numbers, so chunked launches reset at the
  same steps as one launch; ff_reset replays the same sequence.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from paper_1505_00344_gb300.workloads import LORENZ_PARAMS, WC_PARAMS  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()


def G(count, lo, hi, direction, seed):
    return dict(count=count, lo=list(lo), hi=list(hi), direction=direction, seed=seed)


def build(rhs, params, groups, dim, kahan=False, ppt=None):
    s = ff.System(rhs, params, sum(g["count"] for g in groups), dim=dim, kahan=kahan,
                  stream=torch.cuda.current_stream().cuda_stream)
    for g in groups:
        s.seed(g["count"], g["lo"], g["hi"], g["direction"], g["seed"])
    if ppt:
        s.set_launch(ppt)
    return s


def gpu_state(s):
    n, _, dim, _ = s.info()
    x = np.empty((dim, n), np.float32)
    s.get_state(x)
    age = np.empty(n, np.uint32)
    res = np.empty(n, np.uint32)
    s.get_reset_state(age, res)
    return x, age, res


def particle_err(got, want):
    """Per-particle relative state error: max over components k of
    |x_k - x_ref,k| / max(|x_ref,k|, 1) (each component on its own scale, floored at 1)."""
    d = np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1.0)
    return d.max(axis=0)


def oracle_x0(groups, dim):
    return np.concatenate([oracle.seed_group(dim, g["lo"], g["hi"], g["seed"], count=g["count"]) for g in groups],
                          axis=1)


@pytest.mark.parametrize("rhs,params,dim,box,dt,ppt,kahan", [
    ("wilson_cowan", WC_PARAMS, 2, ([0, 0], [1, 1]), 0.01, None, False),
    ("wilson_cowan", WC_PARAMS, 2, ([0, 0], [1, 1]), 0.01, 4, True),
    ("lorenz", LORENZ_PARAMS, 3, ([-30, -30, 0], [30, 30, 60]), 0.001, None, False),
    ("lorenz", LORENZ_PARAMS, 3, ([-30, -30, 0], [30, 30, 60]), 0.001, 2, True),
])
def test_age_limit_resets_exact(rhs, params, dim, box, dt, ppt, kahan):
    groups = [G(1001, *box, 1, 21), G(503, *box, -1, 22)]
    s = build(rhs, params, groups, dim, kahan=kahan, ppt=ppt)
    s.set_reset(None, None, t_max=30 * dt, check_every=1)  # reset every 30 steps
    s.step(100, dt)
    x, age, res = gpu_state(s)
    want, oage, ores = oracle.integrate_reset(ff.RHS_BY_NAME[rhs], oracle_x0(groups, dim), params, groups, dt, 100,
                                              max_age=30)
    np.testing.assert_array_equal(age, oage)
    np.testing.assert_array_equal(res, ores)
    assert (res == 3).all() and (age == 10).all()
    assert particle_err(x, want).max() <= TOL


def test_bounds_resets_backward_wilson_cowan():
    # the paper's pink particles: integrated backward they leave [0,1]^2 and are reset constantly
    box = ([0, 0], [1, 1])
    groups = [G(2048, *box, 1, 31), G(2048, *box, -1, 32)]
    s = build("wilson_cowan", WC_PARAMS, groups, 2)
    s.set_reset([0.0, 0.0], [1.0, 1.0], t_max=5.0, check_every=1)
    s.step(300, 0.01)
    x, age, res = gpu_state(s)
    want, oage, ores = oracle.integrate_reset(oracle.WILSON_COWAN, oracle_x0(groups, 2), WC_PARAMS, groups, 0.01,
                                              300, bounds=([0.0, 0.0], [1.0, 1.0]), max_age=500)
    same = (age == oage) & (res == ores)
    assert same.mean() >= 0.99
    assert res[2048:].mean() > 1.0 and res[:2048].max() == 0  # backward group resets, forward does not
    assert particle_err(x[:, same], want[:, same]).max() <= TOL


@pytest.mark.parametrize("check_every,chunk", [(1, 7), (7, 5), (10, 10)])
def test_schedule_is_global_across_chunks(check_every, chunk):
    box = ([0, 0], [1, 1])
    groups = [G(999, *box, -1, 41)]
    a = build("wilson_cowan", WC_PARAMS, groups, 2)
    b = build("wilson_cowan", WC_PARAMS, groups, 2)
    for s in (a, b):
        s.set_reset([0.0, 0.0], [1.0, 1.0], t_max=0.5, check_every=check_every)
    b.set_launch(1, 128, 0, chunk)
    a.step(120, 0.01)
    for _ in range(4):
        b.step(30, 0.01)
    xa, aa, ra = gpu_state(a)
    xb, ab, rb = gpu_state(b)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(aa, ab)
    np.testing.assert_array_equal(ra, rb)
    want, oage, ores = oracle.integrate_reset(oracle.WILSON_COWAN, oracle_x0(groups, 2), WC_PARAMS, groups, 0.01,
                                              120, check_every=check_every, bounds=([0.0, 0.0], [1.0, 1.0]),
                                              max_age=50)
    assert ((aa == oage) & (ra == ores)).mean() >= 0.99


def test_reset_replays_and_set_state_clears_ages():
    box = ([-30, -30, 0], [30, 30, 60])
    groups = [G(3000, *box, -1, 51)]
    s = build("lorenz", LORENZ_PARAMS, groups, 3)
    s.set_reset([-40.0, -40.0, -20.0], [40.0, 40.0, 80.0], t_max=0.0, check_every=4)
    s.step(500, 0.001)
    x1, a1, r1 = gpu_state(s)
    assert r1.sum() > 0  # backward Lorenz particles leave the box
    s.reset()
    s.step(500, 0.001)
    x2, a2, r2 = gpu_state(s)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(r1, r2)
    s.set_state(x2)
    _, a3, r3 = gpu_state(s)
    assert a3.max() == 0 and r3.max() == 0
    s.set_reset(check_every=0)  # off: no further resets
    s.step(100, 0.001)
    _, _, r4 = gpu_state(s)
    assert r4.max() == 0


def test_reset_argument_errors():
    s = build("lorenz", LORENZ_PARAMS, [G(10, [0, 0, 0], [1, 1, 1], 1, 1)], 3)
    with pytest.raises(ff.FFError):
        s.set_reset([0.0] * 3, None)
    with pytest.raises(ff.FFError):
        s.set_reset([1.0] * 3, [0.0] * 3)
    with pytest.raises(ff.FFError):
        s.set_reset(check_every=-1)
    with pytest.raises(ff.FFError) as e:
        s.get_reset_state(np.empty(10, np.uint32))
    assert e.value.status == ff.FF_ERR_STATE
