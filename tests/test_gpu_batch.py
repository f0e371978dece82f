"""Batched stepping (ff_batch_*): several systems of different right-hand sides in one
graph-captured launch per family.

The batch runs the same per-particle arithmetic as each system's own scalar
integrator, so every member must end bit-identical to the same system stepped
alone with one particle per thread -- across graph replays, a new step count, a
mid-run parameter change and autotuning (which restores the members' states; if it
splits a call into several launches, Lorenz members agree to the rounding of the
shifted state at launch boundaries instead).
Every member is also checked directly against the FP64 oracle over the first 100
steps, at the bar of the single-system parity tests: per-component relative error
|x - x_ref| / max(|x_ref|, 1) <= 1e-5, and for the chaotic systems (Lorenz, HH x 3)
the yardsticks of conftest.assert_parity_bar (the oracle's own one-ulp sensitivity and
an FP32 evaluation of the oracle's formulas).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from conftest import assert_parity_bar, state_err  # noqa: E402
from paper_1505_00344_gb300.workloads import HH3_BASE, LORENZ_PARAMS, WC_PARAMS  # noqa: E402

pytestmark = pytest.mark.gpu
LZ = ([-30, -30, 0], [30, 30, 60])
HHB = ([-80, 0, 0, 0, 0] * 3, [40, 1, 1, 1, 1] * 3)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()


def hh(gsyn):
    p = list(HH3_BASE)
    p[7] = gsyn
    return p


MEMBERS = [  # rhs, params, groups (count, direction), box, dt, per-particle (index, lo, hi)
    ("lorenz", LORENZ_PARAMS, [(3001, 1), (999, -1)], LZ, 0.001, None),
    ("lorenz", LORENZ_PARAMS, [(2048, 1)], LZ, 0.001, (1, 0.0, 60.0)),
    ("wilson_cowan", WC_PARAMS, [(1500, 1), (500, -1)], ([0, 0], [1, 1]), 0.01, None),
    ("hh3", hh(0.2), [(700, 1)], HHB, 0.01, None),
    ("hh3", hh(0.8), [(301, 1)], HHB, 0.01, None),
    ("harmonic", [1.7], [(99, 1)], ([-1, -1], [1, 1]), 0.02, None),
    ("linear", [-0.5, 1.0, 0.0, -1.0, -0.5, 0.2, 0.0, 0.3, -0.9], [(50, 1), (3, -1)], ([-1] * 3, [1] * 3), 0.01,
     None),
]


def make(member, seed, ppt=1):
    rhs, params, groups, box, dt, pp = member
    dim = len(box[0])
    s = ff.System(rhs, params, sum(c for c, _ in groups), dim=dim, stream=torch.cuda.current_stream().cuda_stream)
    for t, (c, d) in enumerate(groups):
        s.seed(c, box[0], box[1], d, seed + t)
    if pp:
        s.set_particle_param(*pp)
    s.set_launch(ppt)
    return s


def state(s):
    n, _, dim, _ = s.info()
    x = np.empty((dim, n), np.float32)
    s.get_state(x)
    return x


def test_batch_matches_members_stepped_alone():
    batched = [make(m, 100 + 10 * i) for i, m in enumerate(MEMBERS)]
    alone = [make(m, 100 + 10 * i) for i, m in enumerate(MEMBERS)]
    dts = [m[4] for m in MEMBERS]
    b = ff.Batch(batched, stream=torch.cuda.current_stream().cuda_stream)
    for n in (60, 60, 37):  # replay, replay, new step count (new capture)
        b.step(n, dts)
        for s, dt in zip(alone, dts):
            s.step(n, dt)
    for i, (x, y) in enumerate(zip(batched, alone)):
        np.testing.assert_array_equal(state(x), state(y), err_msg=f"member {i}")
    # a parameter change between batch steps takes effect at the next one
    batched[0].set_params([10.0, 28.0, 2.0])
    alone[0].set_params([10.0, 28.0, 2.0])
    b.step(20, dts)
    for s, dt in zip(alone, dts):
        s.step(20, dt)
    np.testing.assert_array_equal(state(batched[0]), state(alone[0]))
    # member 2 (Wilson-Cowan) against the oracle over the whole run (177 steps)
    rhs, params, groups, box, dt, _ = MEMBERS[2]
    x0 = np.concatenate([oracle.seed_group(2, box[0], box[1], 120 + t, count=c) for t, (c, _) in enumerate(groups)],
                        axis=1)
    h = np.concatenate([np.full(c, d * dt) for c, d in groups])
    want = oracle.integrate(oracle.WILSON_COWAN, x0, params, h, 177)
    got = state(batched[2]).astype(np.float64)
    err = np.abs(got - want).max(axis=0) / np.maximum(np.abs(want).max(axis=0), 1.0)
    assert err.max() <= 1e-5
    n_esc, t_fwd, t_bwd = batched[2].stats()
    assert abs(t_fwd - 1.77) < 1e-12 and abs(t_bwd + 1.77) < 1e-12
    b.close()


CHAOTIC = {"lorenz", "hh3"}
ORACLE_IDS = {"lorenz": oracle.LORENZ, "wilson_cowan": oracle.WILSON_COWAN, "hh3": oracle.HH3,
              "harmonic": oracle.HARMONIC, "linear": oracle.LINEAR}


@pytest.mark.parametrize("tuned", [False, True])
def test_batch_members_against_oracle(tuned):
    """Each member of one batch (two Lorenz systems, one with a per-particle r; Wilson-Cowan;
    two HH x 3 systems; harmonic; linear) after 100 batched steps against oracle.integrate,
    in the default launch shape (one particle per thread) and in the autotuned one."""
    seed0 = 300 + 17 * int(tuned)
    members = [make(m, seed0 + 10 * i) for i, m in enumerate(MEMBERS)]
    dts = [m[4] for m in MEMBERS]
    b = ff.Batch(members, stream=torch.cuda.current_stream().cuda_stream)
    if tuned:
        b.autotune(dts, trial_steps=16)  # restores the members' states afterwards
    b.step(60, dts)
    b.step(40, dts)  # a second capture: the members carry their states between launches
    for i, (m, s) in enumerate(zip(MEMBERS, members)):
        rhs, params, groups, box, dt, pp = m
        dim = len(box[0])
        x0 = np.concatenate([oracle.seed_group(dim, box[0], box[1], seed0 + 10 * i + t, count=c)
                             for t, (c, _) in enumerate(groups)], axis=1)
        h = np.concatenate([np.full(c, d * dt) for c, d in groups])
        kw = {}
        if pp:
            kw = dict(pparam_index=pp[0], pparam=oracle.linspace_param(x0.shape[1], pp[1], pp[2]).astype(np.float64))
        rid = ORACLE_IDS[rhs]
        want = oracle.integrate(rid, x0, params, h, 100, **kw)
        err = state_err(state(s), want)
        if rhs not in CHAOTIC:
            assert_parity_bar(err)
            continue
        sign = np.random.default_rng(i).choice([-1.0, 1.0], x0.shape)
        pert = oracle.integrate(rid, x0.astype(np.float64) * (1.0 + 6e-8 * sign), params, h, 100, **kw)
        fp32 = oracle.integrate_fp32(rid, x0, params, h, 100, **kw)
        assert_parity_bar(err, state_err(pert, want), h < 0, state_err(fp32, want))
    b.close()


def test_autotune_restores_state_and_keeps_results():
    batched = [make(m, 200 + 10 * i) for i, m in enumerate(MEMBERS)]
    alone = [make(m, 200 + 10 * i) for i, m in enumerate(MEMBERS)]
    dts = [m[4] for m in MEMBERS]
    b = ff.Batch(batched, stream=torch.cuda.current_stream().cuda_stream)
    before = [state(s) for s in batched]
    b.autotune(dts, trial_steps=16)
    for x, y in zip(before, batched):
        np.testing.assert_array_equal(x, state(y))
    text = b.describe()
    assert "lorenz/rk4: 1 systems" in text and "lorenz/rk4/per-particle: 1 systems" in text
    assert "tuned" in text and "untuned" not in text
    b.step(50, dts)
    for s, dt in zip(alone, dts):
        s.step(50, dt)
    for i, (x, y) in enumerate(zip(batched, alone)):
        if MEMBERS[i][0] == "lorenz":
            # the tuner may split the 50 steps into several launches; the Lorenz kernel rounds
            # its shifted state (z - r) at each launch boundary
            np.testing.assert_allclose(state(x), state(y), rtol=2e-6, atol=2e-6, err_msg=f"member {i}")
        else:
            np.testing.assert_array_equal(state(x), state(y), err_msg=f"member {i}")
    b.close()


def test_batch_errors():
    st = torch.cuda.current_stream().cuda_stream
    a = make(MEMBERS[0], 1)
    k = ff.System("lorenz", LORENZ_PARAMS, 10, kahan=True, stream=st)
    k.seed(10, *LZ, 1, 1)
    with pytest.raises(ff.FFError) as e:
        ff.Batch([a, k], stream=st)
    assert e.value.status == ff.FF_ERR_UNSUPPORTED
    with pytest.raises(ff.FFError) as e:
        ff.Batch([a, a], stream=st)
    assert e.value.status == ff.FF_ERR_INVALID_ARG
    c = ff.System("lorenz", LORENZ_PARAMS, 100, stream=st)
    c.seed(10, *LZ, 1, 1)
    b = ff.Batch([a, c], stream=st)
    c.seed(10, *LZ, 1, 2)  # membership changed behind the batch's back
    with pytest.raises(ff.FFError) as e:
        b.step(5, [0.001, 0.001])
    assert e.value.status == ff.FF_ERR_STATE
    b.close()
