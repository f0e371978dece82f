"""Batched gradients: ff_batch_tape_begin / ff_batch_step / ff_batch_backward.

* Every member's taped batch run and reverse sweep match the same system taped
  and swept alone: states and dL/dx0 bit-identical; dL/dp within 1e-8 relative
  (the same per-particle arithmetic compiled into two kernels: their FP64 sums run
  in another order, and one measured case had a single particle's contribution one
  FP32 ulp apart, 1.3e-9 of the sum), across a mid-run parameter change and with a
  per-particle parameter.
* A scaled copy of the differentiable mixed ensemble (Wilson-Cowan, Lorenz and HH3
  systems with uneven particle counts, loss sum_s (1/P_s) sum_i |x_i(T) - t_i|^2)
  against the oracle's forward-sensitivity gradients, member by member, and one
  small member against FP64 central differences of the oracle's loss (h = 1e-3).
Bars as for ff_backward: |g - g_ref| <= 1e-3 max(|g_ref|, 1e-3 max|g_ref|).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from paper_1505_00344_gb300.workloads import HH3_BASE, LORENZ_PARAMS, WC_PARAMS, random_states  # noqa: E402

pytestmark = pytest.mark.gpu
LZ = ([-20, -20, 0], [20, 20, 40])
WCB = ([0, 0], [1, 1])
HHB = ([-80, 0, 0, 0, 0] * 3, [40, 1, 1, 1, 1] * 3)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()


def stream():
    return torch.cuda.current_stream().cuda_stream


def make(rhs, params, groups, box, pp=None):
    dim = len(box[0])
    s = ff.System(rhs, params, sum(c for c, _, _ in groups), dim=dim, stream=stream())
    for c, d, seed in groups:
        s.seed(c, box[0], box[1], d, seed)
    if pp:
        s.set_particle_param(*pp)
    s.set_launch(1)  # the batch runs the one-particle-per-thread integrator
    return s


def check(g, ref):
    bound = 1e-3 * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    worst = float((np.abs(g - ref) / bound).max())
    assert worst <= 1.0, worst


MEMBERS = [  # rhs, params, groups (count, direction, seed), box, dt, per-particle
    ("lorenz", LORENZ_PARAMS, [(301, 1, 5), (99, -1, 6)], LZ, 0.001, None),
    ("lorenz", LORENZ_PARAMS, [(256, 1, 7)], LZ, 0.001, (1, 0.0, 40.0)),
    ("wilson_cowan", WC_PARAMS, [(200, 1, 8), (57, -1, 9)], WCB, 0.01, None),
    ("hh3", HH3_BASE, [(130, 1, 10)], HHB, 0.01, None),
    ("harmonic", [1.7], [(77, 1, 11)], ([-1, -1], [1, 1]), 0.02, None),
    ("linear", [-0.5, 1.0, 0.0, -1.0, -0.5, 0.2, 0.0, 0.3, -0.9], [(50, 1, 12)], ([-1] * 3, [1] * 3), 0.01, None),
]


def targets(s, seed):
    n, _, dim, _ = s.info()
    return torch.from_numpy(random_states(dim, n, [-1.0] * dim, [1.0] * dim, seed=seed)).cuda()


def loss_grad(s, t):
    n, _, dim, _ = s.info()
    x = torch.empty((dim, n), dtype=torch.float32, device="cuda")
    s.get_state(x)
    return (2.0 / n) * (x - t)


def test_batch_backward_matches_members_alone():
    batched = [make(m[0], m[1], m[2], m[3], m[5]) for m in MEMBERS]
    alone = [make(m[0], m[1], m[2], m[3], m[5]) for m in MEMBERS]
    dts = [m[4] for m in MEMBERS]
    b = ff.Batch(batched, stream=stream())
    b.tape_begin(40, 200)
    for s in alone:
        s.tape_begin(40, 200)
    # the parameter change falls on a checkpoint step, so every member's launches split
    # where its own ff_step would split them (a Lorenz launch boundary rounds its
    # shifted state, so other splits are not bit-identical: see the next test)
    b.step(80, dts)
    for s, dt in zip(alone, dts):
        s.step(80, dt)
    batched[0].set_params([10.0, 24.0, 2.5])
    alone[0].set_params([10.0, 24.0, 2.5])
    b.step(45, dts)
    for s, dt in zip(alone, dts):
        s.step(45, dt)
    gb = [loss_grad(s, targets(s, 30 + i)) for i, s in enumerate(batched)]
    ga = [loss_grad(s, targets(s, 30 + i)) for i, s in enumerate(alone)]
    for i in range(len(MEMBERS)):
        torch.testing.assert_close(gb[i], ga[i], rtol=0, atol=0, msg=f"state of member {i}")
    out_b = [torch.empty_like(g) for g in gb]
    dp_b = b.backward(gb, out_b)
    for i, (s, g) in enumerate(zip(alone, ga)):
        out = torch.empty_like(g)
        dp = s.backward(g, out, len(MEMBERS[i][1]))
        torch.testing.assert_close(out_b[i], out, rtol=0, atol=0, msg=f"dL/dx0 of member {i}")
        n_p = len(MEMBERS[i][1])
        np.testing.assert_allclose(dp_b[i, :n_p], dp, rtol=1e-8, atol=1e-11 * np.abs(dp).max(),
                                   err_msg=f"dL/dp of member {i}")
        assert not dp_b[i, n_p:].any()
    b.tape_end()
    b.close()


def test_hh3_members_with_per_particle_parameter_match_alone():
    # the HH3 family's sweep with a per-particle parameter (g_syn linspace; the two members
    # differ in their range and sizes, the second not a multiple of the 80-particle tile)
    spec = [(HH3_BASE, [(150, 1, 21)], (7, 0.0, 1.0)), (HH3_BASE, [(97, 1, 22)], (7, 0.2, 0.6))]
    batched = [make("hh3", p, g, HHB, pp) for p, g, pp in spec]
    alone = [make("hh3", p, g, HHB, pp) for p, g, pp in spec]
    b = ff.Batch(batched, stream=stream())
    b.tape_begin(25, 60)
    for s in alone:
        s.tape_begin(25, 60)
    b.step(60, [0.01, 0.01])
    for s in alone:
        s.step(60, 0.01)
    gb = [loss_grad(s, targets(s, 40 + i)) for i, s in enumerate(batched)]
    ga = [loss_grad(s, targets(s, 40 + i)) for i, s in enumerate(alone)]
    out_b = [torch.empty_like(g) for g in gb]
    dp_b = b.backward(gb, out_b)
    for i, (s, g) in enumerate(zip(alone, ga)):
        torch.testing.assert_close(gb[i], g, rtol=0, atol=0, msg=f"state of member {i}")
        out = torch.empty_like(g)
        dp = s.backward(g, out, 16)
        torch.testing.assert_close(out_b[i], out, rtol=0, atol=0, msg=f"dL/dx0 of member {i}")
        np.testing.assert_allclose(dp_b[i, :16], dp, rtol=1e-8, atol=1e-11 * np.abs(dp).max(),
                                   err_msg=f"dL/dp of member {i}")
    b.tape_end()
    b.close()


def test_parameter_change_between_checkpoints():
    # member 0 (Lorenz, per-particle r) changes beta after 70 steps, off the K = 40 grid:
    # a new chunk for member 0 only, while the others' chunks run on
    members = [MEMBERS[1], MEMBERS[2], MEMBERS[3]]
    batched = [make(m[0], m[1], m[2], m[3], m[5]) for m in members]
    alone = [make(m[0], m[1], m[2], m[3], m[5]) for m in members]
    dts = [m[4] for m in members]
    b = ff.Batch(batched, stream=stream())
    b.tape_begin(40, 200)
    for s in alone:
        s.tape_begin(40, 200)
    n1, n2 = 70, 55
    p2 = [10.0, 28.0, 2.0]
    b.step(n1, dts)
    batched[0].set_params(p2)
    b.step(n2, dts)
    for s, dt in zip(alone, dts):
        s.step(n1, dt)
    alone[0].set_params(p2)
    for s, dt in zip(alone, dts):
        s.step(n2, dt)
    P = 256
    t = random_states(3, P, [-20, -20, 0], [20, 20, 40], seed=61).astype(np.float64)
    g0 = loss_grad(batched[0], torch.from_numpy(t.astype(np.float32)).cuda())
    grads = [g0] + [loss_grad(s, targets(s, 62 + i)) for i, s in enumerate(batched[1:])]
    outs = [torch.empty_like(g) for g in grads]
    dp = b.backward(grads, outs)
    # member 0 against the oracle: sensitivities of the two segments composed
    r = oracle.linspace_param(P, 0.0, 40.0).astype(np.float64)
    x0 = oracle.seed_group(3, LZ[0], LZ[1], 7, count=P).astype(np.float64)
    x1, S1, Q1 = oracle.tangent(oracle.LORENZ, x0, LORENZ_PARAMS, 0.001, n1, pparam_index=1, pparam=r)
    x2, S2, Q2 = oracle.tangent(oracle.LORENZ, x1, p2, 0.001, n2, pparam_index=1, pparam=r)
    g = (2.0 / P) * (x2 - t)
    S = np.einsum("pij,pjk->pik", S2, S1)
    Q = np.einsum("pij,pjq->piq", S2, Q1) + Q2
    check(outs[0].cpu().numpy().astype(np.float64), np.einsum("pij,ip->jp", S, g))
    check(dp[0, :3], np.einsum("piq,ip->q", Q, g))
    # the other members split where they would alone: bit-identical
    for i in (1, 2):
        ga = loss_grad(alone[i], targets(alone[i], 62 + i - 1))
        torch.testing.assert_close(grads[i], ga, rtol=0, atol=0)
        out = torch.empty_like(ga)
        dpa = alone[i].backward(ga, out, len(members[i][1]))
        torch.testing.assert_close(outs[i], out, rtol=0, atol=0)
        np.testing.assert_allclose(dp[i, :len(members[i][1])], dpa, rtol=1e-8, atol=1e-11 * np.abs(dpa).max())
    b.tape_end()
    b.close()


def mixed_members(rng):
    # the mixed ensemble's recipe at reduced sizes: system s has type s mod 3 and a
    # log-uniform particle count; WC dt 0.01, Lorenz dt 0.001, HH3 dt 0.01 ms
    out = []
    for k in range(9):
        n = int(round(np.exp(rng.uniform(np.log(16), np.log(300)))))
        t = k % 3
        if t == 0:
            out.append(("wilson_cowan", WC_PARAMS, [(n, 1, 100 + k)], WCB, 0.01))
        elif t == 1:
            out.append(("lorenz", LORENZ_PARAMS, [(n, 1, 100 + k)], LZ, 0.001))
        else:
            p = list(HH3_BASE)
            p[7] = 0.1 * k
            out.append(("hh3", p, [(n, 1, 100 + k)], HHB, 0.01))
    return out


def test_mixed_ensemble_against_oracle_sensitivities():
    rng = np.random.default_rng(2024)
    members = mixed_members(rng)
    systems = [make(m[0], m[1], m[2], m[3]) for m in members]
    dts = [m[4] for m in members]
    b = ff.Batch(systems, stream=stream())
    n_steps, K = 100, 50  # 1 ms of HH3: the per-particle bars hold (longer spiking runs: test_gpu_adjoint)
    b.tape_begin(K, n_steps)
    b.step(n_steps, dts)
    tg = []
    for i, (s, m) in enumerate(zip(systems, members)):
        n, _, dim, _ = s.info()
        tg.append(random_states(dim, n, m[3][0], m[3][1], seed=500 + i).astype(np.float64))
    grads = [loss_grad(s, torch.from_numpy(t.astype(np.float32)).cuda()) for s, t in zip(systems, tg)]
    outs = [torch.empty_like(g) for g in grads]
    dp = b.backward(grads, outs)
    for i, (m, t) in enumerate(zip(members, tg)):
        rhs, params, groups, box, dt = m
        dim = len(box[0])
        c, _, seed = groups[0]
        x0 = oracle.seed_group(dim, box[0], box[1], seed, count=c).astype(np.float64)
        xT, S, Q = oracle.tangent(ff.RHS_BY_NAME[rhs], x0, params, dt, n_steps)
        g = (2.0 / c) * (xT - t)
        check(outs[i].cpu().numpy().astype(np.float64), np.einsum("pij,ip->jp", S, g))
        per = np.einsum("piq,ip->pq", Q, g)
        ref = per.sum(axis=0)
        check(dp[i, :len(params)], ref)
    b.tape_end()
    b.close()


def test_small_member_against_central_differences():
    members = [("wilson_cowan", WC_PARAMS, [(4, 1, 41)], WCB, 0.01), ("lorenz", LORENZ_PARAMS, [(3, 1, 42)], LZ, 0.001)]
    systems = [make(m[0], m[1], m[2], m[3]) for m in members]
    b = ff.Batch(systems, stream=stream())
    n_steps = 150
    b.tape_begin(50, n_steps)
    b.step(n_steps, [m[4] for m in members])
    rhs, params, groups, box, dt = members[0]
    t = random_states(2, 4, [0, 0], [1, 1], seed=43).astype(np.float64)
    grads = [loss_grad(systems[0], torch.from_numpy(t.astype(np.float32)).cuda()),
             torch.zeros((3, 3), device="cuda")]
    outs = [torch.empty_like(g) for g in grads]
    dp = b.backward(grads, outs)
    x0 = oracle.seed_group(2, box[0], box[1], 41, count=4).astype(np.float64)

    def loss(x, p):
        return float(((oracle.integrate(oracle.WILSON_COWAN, x, p, dt, n_steps) - t) ** 2).sum() / 4)

    h = 1e-3
    fd_x = np.zeros_like(x0)
    for k in range(2):
        for i in range(4):
            e = np.zeros_like(x0)
            e[k, i] = h
            fd_x[k, i] = (loss(x0 + e, params) - loss(x0 - e, params)) / (2 * h)
    fd_p = np.array([(loss(x0, np.add(params, e)) - loss(x0, np.subtract(params, e))) / (2 * h)
                     for e in np.eye(len(params)) * h])
    check(outs[0].cpu().numpy().astype(np.float64), fd_x)
    check(dp[0, :len(params)], fd_p)
    assert not outs[1].any() and not dp[1].any()  # a zero loss gradient gives zero gradients
    b.tape_end()
    b.close()


def test_batch_tape_errors():
    a = make(*MEMBERS[0][:4])
    c = make(*MEMBERS[2][:4])
    b = ff.Batch([a, c], stream=stream())
    g = [torch.zeros((3, 400), device="cuda"), torch.zeros((2, 257), device="cuda")]
    with pytest.raises(ff.FFError) as e:
        b.backward(g, [torch.empty_like(x) for x in g])
    assert e.value.status == ff.FF_ERR_STATE
    b.tape_begin(10, 30)
    with pytest.raises(ff.FFError) as e:
        b.tape_begin(10, 30)
    assert e.value.status == ff.FF_ERR_STATE
    b.step(20, [0.001, 0.01])
    with pytest.raises(ff.FFError) as e:
        b.step(10 * 30, [0.001, 0.01])  # more chunks than the tapes hold
    assert e.value.status == ff.FF_ERR_STATE
    b.tape_end()
    with pytest.raises(ff.FFError) as e:
        b.backward(g, [torch.empty_like(x) for x in g])
    assert e.value.status == ff.FF_ERR_STATE
    b.close()
