"""GPU parity of the hand-written RK4 adjoint (ff_tape_begin / ff_step / ff_backward).

Loss L = (1/P) sum_i |x_i(T) - t_i|^2 with seeded targets.  Reference gradients come
from the oracle's forward sensitivities (RK4 applied to the variational system is
exactly the derivative of the discrete RK4 map) and, on a small case, from FP64
central differences with h = 1e-3.  Bar: |g - g_ref| <= 1e-3 max(|g_ref|,
1e-3 max|g_ref|) for every component of dL/dx0 and dL/dp.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from paper_1505_00344_gb300.workloads import HH3_BASE, LORENZ_PARAMS, WC_PARAMS, random_states  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()


def G(count, lo, hi, direction, seed):
    return dict(count=count, lo=list(lo), hi=list(hi), direction=direction, seed=seed)


def build(rhs, params, groups, dim, method="rk4"):
    s = ff.System(rhs, params, sum(g["count"] for g in groups), dim=dim, method=method,
                  stream=torch.cuda.current_stream().cuda_stream)
    for g in groups:
        s.seed(g["count"], g["lo"], g["hi"], g["direction"], g["seed"])
    return s


def x0_of(groups, dim):
    return np.concatenate([oracle.seed_group(dim, g["lo"], g["hi"], g["seed"], count=g["count"]) for g in groups],
                          axis=1)


def h_of(groups, dt):
    return np.concatenate([np.full(g["count"], g["direction"] * dt) for g in groups])


def gpu_grads(s, dim, P, target, n_params):
    xT = torch.empty((dim, P), dtype=torch.float32, device="cuda")
    s.get_state(xT)
    t = torch.from_numpy(target.astype(np.float32)).cuda()
    g = (2.0 / P) * (xT - t)
    dx0 = torch.empty_like(g)
    dp = s.backward(g, dx0, n_params)
    torch.cuda.synchronize()
    return dx0.cpu().numpy().astype(np.float64), dp


def check(g, ref):
    bound = 1e-3 * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    worst = float((np.abs(g - ref) / bound).max())
    assert worst <= 1.0, worst


HHB = ([-80, 0, 0, 0, 0] * 3, [40, 1, 1, 1, 1] * 3)
CASES = [
    ("lorenz", LORENZ_PARAMS, 3, ([-20, -20, 0], [20, 20, 40]), 0.001, 300, 100, "rk4"),
    ("lorenz", LORENZ_PARAMS, 3, ([-20, -20, 0], [20, 20, 40]), 0.001, 250, 37, "rk4"),
    ("lorenz", LORENZ_PARAMS, 3, ([-20, -20, 0], [20, 20, 40]), 0.0005, 200, 16, "euler"),
    ("wilson_cowan", WC_PARAMS, 2, ([0, 0], [1, 1]), 0.01, 200, 64, "rk4"),
    ("harmonic", [2.5], 2, ([-1, -1], [1, 1]), 0.01, 300, 100, "rk4"),
    ("linear", list((np.arange(9) * 0.37 % 1.0) - 0.5 - np.eye(3).reshape(-1)), 3, ([-1] * 3, [1] * 3), 0.02, 120,
     50, "rk4"),
    # three HH neurons over 1 ms; forward groups only, backward HH is unstable
    ("hh3", HH3_BASE, 15, HHB, 0.01, 100, 50, "rk4"),
    ("hh3", HH3_BASE, 15, HHB, 0.005, 90, 16, "euler"),
]


@pytest.mark.parametrize("rhs,params,dim,box,dt,n,K,method", CASES)
def test_adjoint_matches_forward_sensitivities(rhs, params, dim, box, dt, n, K, method):
    if rhs == "hh3":
        groups = [G(200, *box, 1, 61), G(57, *box, 1, 62)]
    else:
        groups = [G(777, *box, 1, 61), G(250, *box, -1, 62)]
    P = sum(g["count"] for g in groups)
    s = build(rhs, params, groups, dim, method)
    s.tape_begin(K, n)
    s.step(n, dt)
    target = random_states(dim, P, box[0], box[1], seed=5).astype(np.float64)
    dx0, dp = gpu_grads(s, dim, P, target, len(params))
    _, dx0_ref, dp_ref = oracle.mse_gradients(ff.RHS_BY_NAME[rhs], x0_of(groups, dim), params, h_of(groups, dt), n,
                                              target, method=oracle.RK4 if method == "rk4" else oracle.EULER)
    check(dx0, dx0_ref)
    check(dp, dp_ref)


def test_hh3_adjoint_through_spikes():
    """2 ms of HH3 dynamics, through spikes.  dL/dx0 meets the per-particle bar.  The
    parameter gradients are sums over particles that cancel (for the drive currents
    sum_i |c_i| is ~30x |sum_i c_i|), and each contribution c_i carries the FP32
    trajectory's error (3.5e-5 relative at 2 ms); so each component of dL/dp is held
    to the sum of the per-particle bars of its contributions, 1e-3 sum_i |c_i|, as
    well as to the plain bar wherever that is the larger."""
    box = HHB
    groups = [G(200, *box, 1, 61), G(57, *box, 1, 62)]
    P, dt, n = 257, 0.01, 200
    s = build("hh3", HH3_BASE, groups, 15)
    s.tape_begin(100, n)
    s.step(n, dt)
    target = random_states(15, P, box[0], box[1], seed=5).astype(np.float64)
    dx0, dp = gpu_grads(s, 15, P, target, 16)
    xT, S, Q = oracle.tangent(oracle.HH3, x0_of(groups, 15), HH3_BASE, dt, n)
    g = (2.0 / P) * (xT - target)
    check(dx0, np.einsum("pij,ip->jp", S, g))
    per = np.einsum("piq,ip->pq", Q, g)  # per-particle contributions c_i to dL/dp
    ref = per.sum(axis=0)
    bound = np.maximum(1e-3 * np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()), 1e-3 * np.abs(per).sum(axis=0))
    worst = float((np.abs(dp - ref) / bound).max())
    assert worst <= 1.0, worst


@pytest.mark.parametrize("pidx,lo,hi,method", [
    (7, 0.0, 1.0, "rk4"),     # g_syn per particle: its FP64 scaling of the E_syn sums is per particle
    (0, 0.8, 1.2, "rk4"),     # C per particle: every 1/C factor of the products and the sums
    (9, 5.0, 15.0, "euler"),  # neuron 0's drive per particle
])
def test_hh3_adjoint_per_particle_parameter(pidx, lo, hi, method):
    """The HH3 sweep with one parameter taken per particle (a linspace), against the
    oracle's forward sensitivities with the same values; its dL/dp entry is the sum
    over particles of the derivatives with respect to their own values."""
    groups = [G(200, *HHB, 1, 61), G(57, *HHB, 1, 62)]
    P, dt, n, K = 257, (0.01 if method == "rk4" else 0.005), 100, 50
    s = build("hh3", HH3_BASE, groups, 15, method)
    s.set_particle_param(pidx, lo, hi)
    s.tape_begin(K, n)
    s.step(n, dt)
    target = random_states(15, P, HHB[0], HHB[1], seed=5).astype(np.float64)
    dx0, dp = gpu_grads(s, 15, P, target, 16)
    pv = oracle.linspace_param(P, lo, hi).astype(np.float64)
    _, dx0_ref, dp_ref = oracle.mse_gradients(oracle.HH3, x0_of(groups, 15), HH3_BASE, dt, n, target,
                                              pparam_index=pidx, pparam=pv,
                                              method=oracle.RK4 if method == "rk4" else oracle.EULER)
    check(dx0, dx0_ref)
    check(dp, dp_ref)


def test_hh3_adjoint_forward_and_backward_groups_in_one_pair():
    """HH3 with a backward-time group over a short horizon (0.2 ms from near the resting
    state; backward HH runs away from most of the box, and from rest within 0.4 ms).
    201 forward + 56 backward particles: particles 200 and 201 share a lane's f32x2
    registers with step sizes of opposite sign."""
    rest = ([-70, 0.02, 0.5, 0.28, 0.0] * 3, [-60, 0.08, 0.65, 0.35, 0.1] * 3)
    groups = [G(201, *HHB, 1, 64), G(56, *rest, -1, 65)]
    P, dt, n = 257, 0.01, 20
    s = build("hh3", HH3_BASE, groups, 15)
    s.tape_begin(8, n)
    s.step(n, dt)
    target = random_states(15, P, HHB[0], HHB[1], seed=8).astype(np.float64)
    dx0, dp = gpu_grads(s, 15, P, target, 16)
    _, dx0_ref, dp_ref = oracle.mse_gradients(oracle.HH3, x0_of(groups, 15), HH3_BASE, h_of(groups, dt), n, target)
    check(dx0, dx0_ref)
    check(dp, dp_ref)


@pytest.mark.parametrize("P", [1, 3, 21])
def test_hh3_adjoint_small_counts(P):
    """Fewer particles than a warp's 20 (three lanes per particle pair), and one more:
    lanes without a particle, a half-filled last pair and a second warp with one particle."""
    groups = [G(P, *HHB, 1, 63)]
    dt, n = 0.01, 40
    s = build("hh3", HH3_BASE, groups, 15)
    s.tape_begin(16, n)
    s.step(n, dt)
    target = random_states(15, P, HHB[0], HHB[1], seed=7).astype(np.float64)
    dx0, dp = gpu_grads(s, 15, P, target, 16)
    _, dx0_ref, dp_ref = oracle.mse_gradients(oracle.HH3, x0_of(groups, 15), HH3_BASE, dt, n, target)
    check(dx0, dx0_ref)
    check(dp, dp_ref)


def test_adjoint_across_parameter_change_and_per_particle_r():
    # r per particle over [0, 40]; beta switched to 2 half-way: two taped segments
    groups = [G(1500, [-20, -20, 0], [20, 20, 40], 1, 71)]
    P, dt, n1 = 1500, 0.001, 150
    s = build("lorenz", LORENZ_PARAMS, groups, 3)
    s.set_particle_param(1, 0.0, 40.0)
    s.tape_begin(100, 2 * n1)
    s.step(n1, dt)
    p2 = [10.0, 28.0, 2.0]
    s.set_params(p2)
    s.step(n1, dt)
    target = random_states(3, P, [-20, -20, 0], [20, 20, 40], seed=6).astype(np.float64)
    dx0, dp = gpu_grads(s, 3, P, target, 3)
    r = oracle.linspace_param(P, 0.0, 40.0).astype(np.float64)
    x0 = x0_of(groups, 3)
    x1, S1, Q1 = oracle.tangent(oracle.LORENZ, x0, LORENZ_PARAMS, dt, n1, pparam_index=1, pparam=r)
    x2, S2, Q2 = oracle.tangent(oracle.LORENZ, x1, p2, dt, n1, pparam_index=1, pparam=r)
    g = (2.0 / P) * (x2 - target)
    S = np.einsum("pij,pjk->pik", S2, S1)
    Q = np.einsum("pij,pjq->piq", S2, Q1) + Q2
    check(dx0, np.einsum("pij,ip->jp", S, g))
    check(dp, np.einsum("piq,ip->q", Q, g))


def test_adjoint_matches_central_differences():
    # FP64 central differences of the oracle's loss with h = 1e-3 on a small system
    groups = [G(8, [-15, -15, 5], [15, 15, 35], 1, 81)]
    P, dt, n = 8, 0.001, 400
    s = build("lorenz", LORENZ_PARAMS, groups, 3)
    s.tape_begin(100, n)
    s.step(n, dt)
    target = random_states(3, P, [-15, -15, 5], [15, 15, 35], seed=9).astype(np.float64)
    dx0, dp = gpu_grads(s, 3, P, target, 3)
    x0 = x0_of(groups, 3).astype(np.float64)

    def loss(x, p):
        xT = oracle.integrate(oracle.LORENZ, x, p, dt, n)
        return float(((xT - target) ** 2).sum() / P)

    hstep = 1e-3
    fd_p = np.array([(loss(x0, np.add(LORENZ_PARAMS, e)) - loss(x0, np.subtract(LORENZ_PARAMS, e))) / (2 * hstep)
                     for e in np.eye(3) * hstep])
    fd_x = np.zeros_like(x0)
    for k in range(3):
        for i in range(P):
            e = np.zeros_like(x0); e[k, i] = hstep
            fd_x[k, i] = (loss(x0 + e, LORENZ_PARAMS) - loss(x0 - e, LORENZ_PARAMS)) / (2 * hstep)
    check(dp, fd_p)
    check(dx0, fd_x)


def test_autograd_function():
    from paper_1505_00344_gb300.autograd import EnsembleRK4

    groups = [G(600, [-20, -20, 0], [20, 20, 40], 1, 91)]
    s = build("lorenz", LORENZ_PARAMS, groups, 3)
    x0 = torch.from_numpy(x0_of(groups, 3)).cuda().requires_grad_(True)
    p = torch.tensor(LORENZ_PARAMS, dtype=torch.float64, requires_grad=True)
    target = torch.from_numpy(random_states(3, 600, [-20, -20, 0], [20, 20, 40], seed=3)).cuda()
    xT = EnsembleRK4.apply(x0, p, s, 200, 0.001, 100)
    loss = ((xT - target) ** 2).sum() / 600
    loss.backward()
    _, dx0_ref, dp_ref = oracle.mse_gradients(oracle.LORENZ, x0_of(groups, 3), LORENZ_PARAMS, 0.001, 200,
                                              target.cpu().numpy().astype(np.float64))
    check(x0.grad.cpu().numpy().astype(np.float64), dx0_ref)
    check(p.grad.numpy(), dp_ref)


@pytest.mark.parametrize("ppt,kahan,n_fwd", [(1, False, 1000), (4, False, 1000), (4, True, 1000), (4, False, 1001)])
def test_checkpoints_inside_launches_match_split_launches(ppt, kahan, n_fwd):
    """The integrator writes a taped run's checkpoints inside its launches, re-basing
    there as a launch boundary would: one 95-step call and the same steps as calls of
    one chunk each give the same states, checkpoints and gradients, bit for bit; so do
    launches capped at 7 steps and calls of 7 steps (checkpoints inside launches).
    Groups of 1000 + 24 run the group-uniform packed kernels, 1001 + 23 the packed
    kernel with per-particle constants."""
    box = ([-20, -20, 0], [20, 20, 40])
    groups = [G(n_fwd, *box, 1, 11), G(1024 - n_fwd, *box, -1, 12)]
    P = sum(g["count"] for g in groups)

    def run(calls, max_steps=0):
        s = ff.System("lorenz", LORENZ_PARAMS, P, kahan=kahan, stream=torch.cuda.current_stream().cuda_stream)
        for g in groups:
            s.seed(g["count"], g["lo"], g["hi"], g["direction"], g["seed"])
        s.set_launch(ppt, 0, 0, max_steps)
        s.tape_begin(10, 200)
        for n in calls:
            s.step(n, 0.001)
        xT = torch.empty((3, P), dtype=torch.float32, device="cuda")
        s.get_state(xT)
        g = xT - 1.0
        dx0 = torch.empty_like(g)
        dp = s.backward(g, dx0, 3)
        torch.cuda.synchronize()
        return xT.cpu().numpy(), dx0.cpu().numpy(), np.asarray(dp)

    one = run([95])
    split = run([10] * 9 + [5])
    np.testing.assert_array_equal(one[0], split[0])
    np.testing.assert_array_equal(one[1], split[1])
    np.testing.assert_allclose(one[2], split[2], rtol=1e-12)
    capped = run([95], max_steps=7)
    sevens = run([7] * 13 + [4])
    np.testing.assert_array_equal(capped[0], sevens[0])
    np.testing.assert_array_equal(capped[1], sevens[1])
    np.testing.assert_allclose(capped[2], sevens[2], rtol=1e-12)
    # re-basing at other places changes only roundings
    assert np.abs(capped[0] - one[0]).max() <= 1e-4 * np.abs(one[0]).max()


def test_tape_errors():
    s = build("lorenz", LORENZ_PARAMS, [G(64, [0, 0, 0], [1, 1, 1], 1, 1)], 3)
    g = torch.zeros((3, 64), device="cuda")
    with pytest.raises(ff.FFError) as e:
        s.backward(g, torch.empty_like(g), 3)
    assert e.value.status == ff.FF_ERR_STATE
    s.tape_begin(10, 20)
    s.step(20, 0.001)
    with pytest.raises(ff.FFError) as e:
        s.step(10 * 20, 0.001)  # more chunks than the tape holds
    assert e.value.status == ff.FF_ERR_STATE
    with pytest.raises(ff.FFError) as e:
        s.set_reset(None, None, 1.0, 1)
    assert e.value.status == ff.FF_ERR_UNSUPPORTED
    s.set_state(np.zeros((3, 64), np.float32))  # ends the tape
    with pytest.raises(ff.FFError):
        s.backward(g, torch.empty_like(g), 3)
    with pytest.raises(ff.FFError):
        s.tape_begin(0, 10)
    r = ff.System("lorenz", LORENZ_PARAMS, 8, stream=torch.cuda.current_stream().cuda_stream)
    r.seed(8, [0] * 3, [1] * 3, 1, 1)
    r.set_reset(None, None, 1.0, 1)
    with pytest.raises(ff.FFError) as e:
        r.tape_begin(10, 10)  # particle reset is not differentiable
    assert e.value.status == ff.FF_ERR_UNSUPPORTED
