"""GPU-vs-oracle parity of every hot-path step, through the C ABI.

* seeding and the per-particle parameter linspace: bit-exact;
* integration (RK4 / Euler, plain / Kahan, 1-2-4 particles per thread, forward
  and backward groups, per-particle parameters, mid-run parameter changes):
  max relative state error <= 1e-5 over the first 100 steps against the FP64
  oracle started from the same FP32 initial conditions, where the error of a
  particle is max_k |x_k - x_ref,k| / max(|x_ref,k|, 1) (each component relative
  to its own magnitude, floored at 1 since gates are ~0-1 and V is tens of mV).
  For the two chaotic systems (Lorenz, whose
  divergence grows with r, and Hodgkin-Huxley, whose spike initiation amplifies
  perturbations) a one-ulp change of the initial state can already move the
  FP64 oracle by about 1e-5 within 100 steps; there the bound is
  max(1e-5, 5 x that one-ulp spread) -- the random-walk size of 100 half-ulp
  roundings -- and 99% of the particles must still be within 1e-5; backward-time
  Lorenz particles (unstable in reverse time) are held to 1e-4;
* projection + splat: bit-exact images against the oracle's FP32 projection of
  the same seeded states (including NaN/inf/huge values, window edges, group
  masks, accumulation, the per-particle parameter axis and 3D cameras);
* escaped-particle counts: exact.
Sizes span several blocks and a ragged tail (particle counts not a multiple of
4, groups of one particle).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from conftest import TOL, assert_parity_bar, state_err  # noqa: E402
from paper_1505_00344_gb300.workloads import (HH3_BASE, LORENZ_PARAMS, WC_PARAMS, hh3_params,  # noqa: E402
                                              look_at_perspective, random_states)

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()  # loud failure if the extension is missing
    torch.cuda.init()


def get_state(sysobj):
    n, _, dim, _ = sysobj.info()
    out = np.empty((dim, n), dtype=np.float32)
    sysobj.get_state(out)
    return out


particle_err = state_err


def rel_err(got, want):
    return float(np.max(particle_err(got, want)))


def oracle_seed(groups, dim):
    """Initial conditions of all groups from the oracle's own seeding."""
    return np.concatenate([oracle.seed_group(dim, g["lo"], g["hi"], g["seed"], count=g["count"])
                           for g in groups], axis=1)


def oracle_h(groups, dt):
    return np.concatenate([np.full(g["count"], g["direction"] * dt) for g in groups])


def make_system(rhs, params, groups, dim, method="rk4", kahan=False, ppt=1, capacity=None):
    cap = capacity or sum(g["count"] for g in groups)
    s = ff.System(rhs, params, cap, dim=dim, method=method, kahan=kahan,
                  stream=torch.cuda.current_stream().cuda_stream)
    for g in groups:
        s.seed(g["count"], g["lo"], g["hi"], g["direction"], g["seed"])
    s.set_launch(particles_per_thread=ppt)
    return s


def G(count, lo, hi, direction, seed):
    return dict(count=count, lo=list(lo), hi=list(hi), direction=direction, seed=seed)


# ---------------------------------------------------------------------------
# seeding
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,counts", [(3, [1]), (3, [1000, 37]), (2, [2048, 2048]), (15, [513, 1, 99]),
                                        (3, [3145728 // 64, 1048576 // 64])])
def test_seed_bit_exact(dim, counts):
    rng = np.random.default_rng(dim * 100 + len(counts))
    groups = []
    for t, c in enumerate(counts):
        lo = rng.uniform(-50, 0, dim)
        hi = lo + rng.uniform(0.0, 80, dim)
        groups.append(G(c, lo, hi, 1 if t % 2 == 0 else -1, 1000 + 77 * t))
    rhs = {2: "wilson_cowan", 3: "lorenz", 15: "hh3"}[dim]
    params = {2: WC_PARAMS, 3: LORENZ_PARAMS, 15: HH3_BASE}[dim]
    s = make_system(rhs, params, groups, dim, capacity=sum(counts) + 5)
    np.testing.assert_array_equal(get_state(s), oracle_seed(groups, dim))
    # reset re-creates exactly the same initial conditions
    s.step(3, 0.001)
    s.reset()
    np.testing.assert_array_equal(get_state(s), oracle_seed(groups, dim))


@pytest.mark.parametrize("P", [1, 2, 1023, 8191])
def test_linspace_bit_exact(P):
    s = make_system("lorenz", LORENZ_PARAMS, [G(P, [-20, -20, 0], [20, 20, 40], 1, 5)], 3)
    s.set_particle_param(1, 0.0, 200.0)
    got = np.empty(P, dtype=np.float32)
    assert s.get_particle_param(got) == 1
    np.testing.assert_array_equal(got, oracle.linspace_param(P, 0.0, 200.0))


# ---------------------------------------------------------------------------
# integration parity over the first 100 steps
# ---------------------------------------------------------------------------
LZ_BOX = ([-30, -30, 0], [30, 30, 60])
CASES = {
    "lorenz": ("lorenz", LORENZ_PARAMS, 3, LZ_BOX, 0.001),
    "wc": ("wilson_cowan", WC_PARAMS, 2, ([0, 0], [1, 1]), 0.01),
    "hh3": ("hh3", hh3_params(), 15, ([-80, 0, 0, 0, 0] * 3, [40, 1, 1, 1, 1] * 3), 0.01),
    "harmonic": ("harmonic", [2.5], 2, ([-1, -1], [1, 1]), 0.01),
}


CHAOTIC = {oracle.LORENZ, oracle.HH3}


def check_parity(rid, got, want, x0, params, h, steps, method=0, **kw):
    """The parity bar (conftest.assert_parity_bar): 1e-5 per component; for the chaotic
    systems the one-ulp-sensitivity and FP32-evaluation yardsticks, forward and backward
    particles apart."""
    err = particle_err(got, want)
    if rid not in CHAOTIC:
        return assert_parity_bar(err)
    sign = np.random.default_rng(0).choice([-1.0, 1.0], x0.shape)
    pert = oracle.integrate(rid, x0.astype(np.float64) * (1.0 + 6e-8 * sign), params, h, steps, method=method, **kw)
    fp32 = oracle.integrate_fp32(rid, x0, params, h, steps, method=method, **kw)
    backward = np.broadcast_to(np.asarray(h, dtype=np.float64), (x0.shape[1],)) < 0
    return assert_parity_bar(err, particle_err(pert, want), backward, particle_err(fp32, want))


def _run_case(name, method, kahan, ppt, counts=(1000, 37), steps=100):
    rhs, params, dim, (lo, hi), dt = CASES[name]
    # Hodgkin-Huxley runs forward only (the paper's HH groups); backward it leaves any bound
    direction = (lambda t: 1) if name == "hh3" else (lambda t: 1 if t % 2 == 0 else -1)
    groups = [G(c, lo, hi, direction(t), 4242 + t) for t, c in enumerate(counts)]
    s = make_system(rhs, params, groups, dim, method=method, kahan=kahan, ppt=ppt)
    s.step(steps, dt)
    got = get_state(s)
    x0 = oracle_seed(groups, dim)
    rid = ff.RHS_BY_NAME[rhs]
    want = oracle.integrate(rid, x0, params, oracle_h(groups, dt), steps,
                            method=oracle.RK4 if method == "rk4" else oracle.EULER)
    return got, want, groups


@pytest.mark.parametrize("name", ["lorenz", "wc", "hh3", "harmonic"])
@pytest.mark.parametrize("method", ["rk4", "euler"])
@pytest.mark.parametrize("kahan", [False, True])
def test_integrate_parity(name, method, kahan):
    got, want, groups = _run_case(name, method, kahan, ppt=1)
    rhs, params, dim, _, dt = CASES[name]
    check_parity(ff.RHS_BY_NAME[rhs], got, want, oracle_seed(groups, dim), params, oracle_h(groups, dt), 100,
                 method=oracle.RK4 if method == "rk4" else oracle.EULER)


@pytest.mark.parametrize("method,kahan", [("rk4", False), ("euler", False), ("rk4", True)])
def test_hh3_two_particles_per_thread_bit_identical(method, kahan):
    """HH x 3 at two particles per thread (RK4: all three neurons of a particle pair packed in
    f32x2, for an ensemble that fills a wave of pairs; Euler and the compensated update fall
    back to one particle per thread) ends bit-identical to one particle per thread -- also for a
    pair that straddles a forward / backward group boundary (lanes with different signed steps)
    and across chunked launches -- and meets the oracle bar on a sample."""
    rhs, params, dim, (lo, hi), dt = CASES["hh3"]
    groups = [G(120_001, lo, hi, 1, 61), G(37, lo, hi, -1, 62), G(2, lo, hi, 1, 63)]
    one = make_system(rhs, params, groups, dim, method=method, kahan=kahan, ppt=1)
    two = make_system(rhs, params, groups, dim, method=method, kahan=kahan, ppt=2)
    chunked = make_system(rhs, params, groups, dim, method=method, kahan=kahan, ppt=2)
    chunked.set_launch(2, 0, 0, 13)
    for sysobj in (one, two, chunked):
        sysobj.step(60, dt)
    np.testing.assert_array_equal(get_state(two), get_state(one))
    np.testing.assert_array_equal(get_state(chunked), get_state(one))
    pair = "hh3_rk4_x2_kernel" in two.last_launch()["kernel"]
    assert pair == (method == "rk4" and not kahan)
    idx = np.sort(np.random.default_rng(8).choice(120_001, 2000, replace=False))
    x0 = oracle_seed(groups, dim)[:, idx]
    h = oracle_h(groups, dt)[idx]
    m = oracle.RK4 if method == "rk4" else oracle.EULER
    want = oracle.integrate(oracle.HH3, x0, params, h, 60, method=m)
    check_parity(oracle.HH3, get_state(two)[:, idx], want, x0, params, h, 60, method=m)


def test_hh3_two_particles_per_thread_small_ensemble_runs_singles():
    rhs, params, dim, (lo, hi), dt = CASES["hh3"]
    s = make_system(rhs, params, [G(16_384, lo, hi, 1, 64)], dim, ppt=2)
    s.step(5, dt)
    assert "integrate_kernel<ff::HH3" in s.last_launch()["kernel"]  # too few pairs to fill a wave


def test_hh3_two_particles_per_thread_taped_checkpoints():
    """A taped HH x 3 run at two particles per thread writes the checkpoints of the run at one
    particle per thread, and the adjoint from them gives the same gradients."""
    rhs, params, dim, (lo, hi), dt = CASES["hh3"]
    n = 120_004
    groups = [G(n, lo, hi, 1, 71)]
    grads = []
    for ppt in (1, 2):
        s = make_system(rhs, params, groups, dim, ppt=ppt)
        s.tape_begin(10, 50)
        s.step(50, dt)
        assert ("hh3_rk4_x2_kernel" in s.last_launch()["kernel"]) == (ppt == 2)
        xT = torch.empty((dim, n), dtype=torch.float32, device="cuda")
        s.get_state(xT)
        g = (xT * 1e-3).contiguous()
        out = torch.empty_like(g)
        dp = s.backward(g, out, len(params))
        grads.append((xT.cpu().numpy(), out.cpu().numpy(), np.asarray(dp)))
        s.tape_end()
    np.testing.assert_array_equal(grads[0][0], grads[1][0])
    np.testing.assert_array_equal(grads[0][1], grads[1][1])
    np.testing.assert_array_equal(grads[0][2], grads[1][2])


def test_hh3_backward_escapes_like_oracle():
    rhs, params, dim, (lo, hi), dt = CASES["hh3"]
    groups = [G(2000, lo, hi, -1, 99)]
    s = make_system(rhs, params, groups, dim)
    s.step(100, dt)
    got = get_state(s)
    want = oracle.integrate(oracle.HH3, oracle_seed(groups, dim), params, -dt, 100)
    esc_gpu = oracle.count_escaped(got.astype(np.float64))[1]
    esc_ref = oracle.count_escaped(want)[1]
    assert (esc_gpu == esc_ref).mean() >= 0.99
    n, _, _ = s.stats()
    assert n == int(esc_gpu.sum())


@pytest.mark.parametrize("name", ["lorenz", "wc", "harmonic"])
@pytest.mark.parametrize("ppt", [2, 4])
@pytest.mark.parametrize("kahan", [False, True])
def test_integrate_parity_vector_width(name, ppt, kahan):
    got, want, groups = _run_case(name, "rk4", kahan, ppt=ppt, counts=(4097, 1, 2, 3))
    rhs, params, dim, _, dt = CASES[name]
    check_parity(ff.RHS_BY_NAME[rhs], got, want, oracle_seed(groups, dim), params, oracle_h(groups, dt), 100)


@pytest.mark.parametrize("ppt", [2, 4])
@pytest.mark.parametrize("r_per_particle", [False, True])
def test_lorenz_group_uniform_kernel(ppt, r_per_particle):
    # every group starts on a multiple of 4: the group-uniform packed kernel runs
    counts = (4096, 1024, 12, 4, 2000)
    groups = [G(c, *LZ_BOX, 1 if t % 2 == 0 else -1, 70 + t) for t, c in enumerate(counts)]
    P = sum(counts)
    s = make_system("lorenz", LORENZ_PARAMS, groups, 3, ppt=ppt)
    kw = {}
    if r_per_particle:
        s.set_particle_param(1, 0.0, 60.0)
        kw = dict(pparam_index=1, pparam=oracle.linspace_param(P, 0.0, 60.0).astype(np.float64))
    s.step(100, 0.001)
    x0 = oracle_seed(groups, 3)
    want = oracle.integrate(oracle.LORENZ, x0, LORENZ_PARAMS, oracle_h(groups, 0.001), 100, **kw)
    check_parity(oracle.LORENZ, get_state(s), want, x0, LORENZ_PARAMS, oracle_h(groups, 0.001), 100, **kw)


@pytest.mark.parametrize("ppt", [1, 2, 4])
@pytest.mark.parametrize("sigma_per_particle", [False, True])
def test_lorenz_other_per_particle_params(ppt, sigma_per_particle):
    # sigma or beta as the per-particle parameter (the packed kernel folds both into constants)
    P = 3001
    groups = [G(2000, *LZ_BOX, 1, 5), G(P - 2000, *LZ_BOX, -1, 6)]
    s = make_system("lorenz", LORENZ_PARAMS, groups, 3, ppt=ppt)
    idx, lo, hi = (0, 5.0, 15.0) if sigma_per_particle else (2, 1.0, 4.0)
    s.set_particle_param(idx, lo, hi)
    s.step(100, 0.001)
    vals = oracle.linspace_param(P, lo, hi).astype(np.float64)
    x0 = oracle_seed(groups, 3)
    want = oracle.integrate(oracle.LORENZ, x0, LORENZ_PARAMS, oracle_h(groups, 0.001), 100,
                            pparam_index=idx, pparam=vals)
    check_parity(oracle.LORENZ, get_state(s), want, x0, LORENZ_PARAMS, oracle_h(groups, 0.001), 100,
                 pparam_index=idx, pparam=vals)


def test_linear_system_parity():
    rng = np.random.default_rng(3)
    for dim in (1, 3, 8):
        A = rng.standard_normal((dim, dim))
        A -= (np.abs(np.linalg.eigvals(A).real).max() + 0.5) * np.eye(dim)
        groups = [G(777, [-1] * dim, [1] * dim, 1, 9), G(5, [-1] * dim, [1] * dim, -1, 10)]
        s = make_system("linear", A.reshape(-1), groups, dim)
        s.step(100, 0.01)
        got = get_state(s)
        want = oracle.integrate(oracle.LINEAR, oracle_seed(groups, dim), A.reshape(-1),
                                oracle_h(groups, 0.01), 100)
        assert rel_err(got, want) <= TOL


@pytest.mark.parametrize("ppt,kahan", [(1, False), (2, False), (4, False), (1, True), (4, True)])
def test_per_particle_param_and_midrun_set_params(ppt, kahan):
    # bifurcation-diagram shape: r per particle over [0, 200]; beta switched to 2 after 50 steps
    P = 6001
    groups = [G(P, [-20, -20, 0], [20, 20, 40], 1, 77)]
    s = make_system("lorenz", LORENZ_PARAMS, groups, 3, ppt=ppt, kahan=kahan)
    s.set_particle_param(1, 0.0, 200.0)
    s.step(50, 0.001)
    s.set_params([10.0, 28.0, 2.0])
    s.step(50, 0.001)
    got = get_state(s)
    r = oracle.linspace_param(P, 0.0, 200.0).astype(np.float64)
    x0 = oracle_seed(groups, 3)

    def two_phase(start):
        y = oracle.integrate(oracle.LORENZ, start, LORENZ_PARAMS, 0.001, 50, pparam_index=1, pparam=r)
        return oracle.integrate(oracle.LORENZ, y, [10.0, 28.0, 2.0], 0.001, 50, pparam_index=1, pparam=r)

    x = two_phase(x0)
    err = particle_err(got, x)
    sign = np.random.default_rng(0).choice([-1.0, 1.0], x0.shape)
    y = oracle.integrate_fp32(oracle.LORENZ, x0, LORENZ_PARAMS, 0.001, 50, pparam_index=1, pparam=r)
    y = oracle.integrate_fp32(oracle.LORENZ, y, [10.0, 28.0, 2.0], 0.001, 50, pparam_index=1, pparam=r)
    assert_parity_bar(err, particle_err(two_phase(x0.astype(np.float64) * (1.0 + 6e-8 * sign)), x), None,
                      particle_err(y, x))
    n, tf, tb = s.stats()
    assert n == 0 and abs(tf - 0.1) < 1e-15 and tb == 0.0


@pytest.mark.parametrize("ppt", [1, 4])
def test_chunked_launches_match_single_launch(ppt):
    rhs, params, dim, (lo, hi), dt = CASES["lorenz"]
    groups = [G(3000, lo, hi, 1, 1), G(1000, lo, hi, -1, 2)]
    a = make_system(rhs, params, groups, dim, ppt=ppt)
    b = make_system(rhs, params, groups, dim, ppt=ppt)
    b.set_launch(ppt, 128, 1, 7)
    a.step(100, dt)
    b.step(100, dt)
    # both within the parity bar of the oracle (the chunks differ from one launch by the
    # rounding of the re-based state at each of the 14 launch boundaries)
    x0 = oracle_seed(groups, dim)
    h = oracle_h(groups, dt)
    want = oracle.integrate(oracle.LORENZ, x0, params, h, 100)
    for sysobj in (a, b):
        check_parity(oracle.LORENZ, get_state(sysobj), want, x0, params, h, 100)
    w = make_system("wilson_cowan", WC_PARAMS, [G(999, [0, 0], [1, 1], 1, 3)], 2)
    v = make_system("wilson_cowan", WC_PARAMS, [G(999, [0, 0], [1, 1], 1, 3)], 2)
    v.set_launch(1, 64, 1, 13)
    w.step(100, 0.01)
    v.step(100, 0.01)
    np.testing.assert_array_equal(get_state(w), get_state(v))  # no re-basing: bit-identical


def test_step_zero_and_state_roundtrip():
    rhs, params, dim, (lo, hi), dt = CASES["wc"]
    s = make_system(rhs, params, [G(10, lo, hi, 1, 3)], dim)
    x0 = get_state(s)
    s.step(0, dt)
    np.testing.assert_array_equal(get_state(s), x0)
    y = random_states(dim, 10, lo, hi, seed=5)
    s.set_state(y)
    np.testing.assert_array_equal(get_state(s), y)
    dev = torch.from_numpy(y * 2).cuda()
    s.set_state(dev)
    out = torch.empty_like(dev)
    s.get_state(out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), y * 2)


# ---------------------------------------------------------------------------
# projection + splat: bit-exact against the oracle's FP32 projection
# ---------------------------------------------------------------------------
def _splat_gpu(s, view, W, H):
    img = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    s.project_splat(view, img)
    torch.cuda.synchronize()
    return img.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n,W,H", [(1, 7, 5), (50_001, 256, 256), (4_194_304, 1920, 1080)])
def test_splat_2d_bit_exact(n, W, H):
    lo, hi = (-30.0, 0.0), (30.0, 60.0)
    x = random_states(3, n, [-35, -40, -5], [35, 40, 65], seed=n, specials=True)
    s = make_system("lorenz", LORENZ_PARAMS, [G(n, [0] * 3, [1] * 3, 1, 1)], 3)
    s.set_state(x)
    view = dict(ndim_view=2, axes=(0, 2), lo=lo, hi=hi, width=W, height=H)
    got = _splat_gpu(s, view, W, H)
    want = oracle.splat2d(x[0], x[2], lo, hi, W, H)
    np.testing.assert_array_equal(got, want)
    # host image path gives the same result
    host = np.zeros((H, W), dtype=np.uint32)
    s.project_splat(view, host)
    np.testing.assert_array_equal(host, want)


def test_splat_narrow_columns_use_shared_histogram_exactly():
    # bifurcation-diagram shape: consecutive particles share a parameter column
    P = 300_000
    x = random_states(3, P, [-20, -20, 0], [20, 20, 80], seed=11)
    s = make_system("lorenz", LORENZ_PARAMS, [G(P, [0] * 3, [1] * 3, 1, 1)], 3)
    s.set_state(x)
    s.set_particle_param(1, 0.0, 200.0)
    r = oracle.linspace_param(P, 0.0, 200.0)
    view = dict(ndim_view=2, axes=(3, 2), lo=(0.0, 0.0), hi=(200.0, 400.0), width=2048, height=1024)
    got = _splat_gpu(s, view, 2048, 1024)
    np.testing.assert_array_equal(got, oracle.splat2d(r, x[2], (0.0, 0.0), (200.0, 400.0), 2048, 1024))
    # a view whose window is a handful of pixels (everything lands in a few bins)
    view = dict(ndim_view=2, axes=(0, 1), lo=(-20.0, -20.0), hi=(20.0, 20.0), width=3, height=2)
    np.testing.assert_array_equal(_splat_gpu(s, view, 3, 2),
                                  oracle.splat2d(x[0], x[1], (-20.0, -20.0), (20.0, 20.0), 3, 2))


def test_splat_group_mask_and_accumulate():
    counts = [1000, 3, 20000]
    groups = [G(c, [-1, -1], [1, 1], 1, 50 + t) for t, c in enumerate(counts)]
    s = make_system("harmonic", [1.0], groups, 2)
    x = get_state(s)
    W, H = 64, 48
    inc = np.zeros(sum(counts), np.uint8)
    inc[:1000] = 1
    inc[1003:] = 1
    view = dict(ndim_view=2, axes=(0, 1), lo=(-1.0, -1.0), hi=(1.0, 1.0), width=W, height=H, group_mask=0b101)
    img = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    s.project_splat(view, img)
    view["accumulate"] = 1
    s.project_splat(view, img)
    torch.cuda.synchronize()
    want = oracle.splat2d(x[0], x[1], (-1, -1), (1, 1), W, H, include=inc)
    np.testing.assert_array_equal(img.cpu().numpy().view(np.uint32), 2 * want)
    view["group_mask"] = 0
    view["accumulate"] = 0
    assert _splat_gpu(s, view, W, H).sum() == 0


@pytest.mark.parametrize("n", [5, 100_003])
def test_splat_3d_bit_exact(n):
    W, H = 1024, 1024
    mvp = look_at_perspective((150.0, 150.0, 150.0), (-20.0, -20.0, -20.0), (0.0, 0.0, 1.0), 45.0, 1.0, 1.0,
                              1000.0)
    x = random_states(15, n, [-100] * 15, [60] * 15, seed=n, specials=True)
    x[[0, 5, 10], 0] = 150.0  # at the camera
    x[[0, 5, 10], min(1, n - 1)] = 200.0  # behind the camera
    s = make_system("hh3", HH3_BASE, [G(n, [0] * 15, [1] * 15, 1, 1)], 15)
    s.set_state(np.ascontiguousarray(x))
    view = dict(ndim_view=3, axes=(0, 5, 10), mvp=mvp, width=W, height=H)
    got = _splat_gpu(s, view, W, H)
    np.testing.assert_array_equal(got, oracle.splat3d(x[0], x[5], x[10], mvp, W, H))


def test_escape_count_exact():
    x = random_states(3, 100_000, [-1, -1, -1], [1, 1, 1], seed=2, specials=True)
    s = make_system("lorenz", LORENZ_PARAMS, [G(100_000, [0] * 3, [1] * 3, 1, 1)], 3)
    s.set_state(x)
    n, _, _ = s.stats()
    assert n == oracle.count_escaped(x)[0] > 0


# ---------------------------------------------------------------------------
# errors that need a live system
# ---------------------------------------------------------------------------
def test_state_errors():
    s = ff.System("lorenz", LORENZ_PARAMS, 100, stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(ff.FFError) as e:
        s.step(1, 0.1)
    assert e.value.status == ff.FF_ERR_STATE
    s.seed(60, LZ_BOX[0], LZ_BOX[1], 1, 1)
    with pytest.raises(ff.FFError) as e:
        s.seed(41, LZ_BOX[0], LZ_BOX[1], 1, 2)  # over capacity
    assert e.value.status == ff.FF_ERR_INVALID_ARG
    with pytest.raises(ff.FFError):
        s.seed(10, LZ_BOX[0], LZ_BOX[1], 0, 2)  # bad direction
    s.step(1, 0.001)
    with pytest.raises(ff.FFError) as e:
        s.seed(10, LZ_BOX[0], LZ_BOX[1], 1, 2)  # after stepping
    assert e.value.status == ff.FF_ERR_STATE
    s.reset()
    s.seed(40, LZ_BOX[0], LZ_BOX[1], -1, 2)
    assert s.info()[0] == 100
    img = torch.zeros((4, 4), dtype=torch.int32, device="cuda")
    for bad in (dict(ndim_view=4), dict(axes=(0, 3)), dict(width=0), dict(lo=(1.0, 0.0), hi=(1.0, 1.0))):
        view = dict(ndim_view=2, axes=(0, 1), lo=(0.0, 0.0), hi=(1.0, 1.0), width=4, height=4)
        view.update(bad)
        with pytest.raises(ff.FFError) as e:
            s.project_splat(view, img)
        assert e.value.status == ff.FF_ERR_INVALID_ARG
    with pytest.raises(ff.FFError):
        s.set_launch(3)
    with pytest.raises(ff.FFError):
        s.step(-1, 0.01)
    with pytest.raises(ff.FFError):
        s.step(1, float("inf"))
    with pytest.raises(ff.FFError):
        s.set_params([1.0, 2.0])
    groups_ok = ff.System("lorenz", LORENZ_PARAMS, 64, stream=torch.cuda.current_stream().cuda_stream)
    for t in range(ff.FF_MAX_GROUPS):
        groups_ok.seed(1, LZ_BOX[0], LZ_BOX[1], 1, t)
    with pytest.raises(ff.FFError) as e:
        groups_ok.seed(1, LZ_BOX[0], LZ_BOX[1], 1, 99)
    assert e.value.status == ff.FF_ERR_STATE


# ---------------------------------------------------------------------------
# ff_step_splat: identical to ff_step + ff_project_splat (fused or not)
# ---------------------------------------------------------------------------
FUSE_VIEWS = {
    "xz": dict(ndim_view=2, axes=(0, 2), lo=(-30.0, 0.0), hi=(30.0, 60.0), width=640, height=360),
    "xz_group1": dict(ndim_view=2, axes=(0, 2), lo=(-30.0, 0.0), hi=(30.0, 60.0), width=640, height=360,
                      group_mask=0b10),
    "cam3d": dict(ndim_view=3, axes=(0, 1, 2), width=300, height=200,
                  mvp=look_at_perspective((60.0, 60.0, 80.0), (0.0, 0.0, 25.0), (0.0, 0.0, 1.0), 50.0, 1.5, 1.0,
                                          500.0)),
    "r_axis": dict(ndim_view=2, axes=(3, 2), lo=(0.0, 0.0), hi=(60.0, 120.0), width=512, height=256),
}


@pytest.mark.parametrize("view_name,counts,ppt,kahan,pp,accumulate", [
    ("xz", (3000, 1000), 4, False, False, False),        # fused
    ("xz_group1", (3000, 1000), 2, False, False, True),  # fused, masked, accumulating
    ("cam3d", (1001,), 4, False, False, False),           # fused, ragged count (padding not drawn)
    ("r_axis", (2048, 1024), 4, False, True, False),      # fused with per-particle r
    ("xz", (3000, 1001), 4, False, False, False),        # ragged total (padded last item): fused
    ("xz", (3001, 1000), 4, False, False, False),        # group start not a multiple of 4: separate calls
    ("xz", (3000, 1000), 4, True, False, False),         # Kahan: separate calls
    ("xz", (3000, 1000), 1, False, False, False),        # scalar kernel: separate calls
])
def test_step_splat_equals_step_then_splat(view_name, counts, ppt, kahan, pp, accumulate):
    view = dict(FUSE_VIEWS[view_name], accumulate=int(accumulate))
    groups = [G(c, *LZ_BOX, 1 if t == 0 else -1, 300 + t) for t, c in enumerate(counts)]
    a = make_system("lorenz", LORENZ_PARAMS, groups, 3, ppt=ppt, kahan=kahan)
    b = make_system("lorenz", LORENZ_PARAMS, groups, 3, ppt=ppt, kahan=kahan)
    if pp:
        a.set_particle_param(1, 0.0, 60.0)
        b.set_particle_param(1, 0.0, 60.0)
    H, W = view["height"], view["width"]
    ia = torch.zeros((H, W), dtype=torch.int32, device="cuda") + (7 if accumulate else 0)
    ib = ia.clone()
    for _ in range(3):
        a.step_splat(150, 0.001, view, ia)
        b.step(150, 0.001)
        b.project_splat(view, ib)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(get_state(a), get_state(b))
    assert torch.equal(ia, ib)
    assert int(ia.sum()) > 0


@pytest.mark.parametrize("counts,ppt,kahan,expect,fused", [
    ((3000, 1000), 4, False, "lorenz_rk4_x2u_kernel<false, 2, true>", True),   # the bench's fused path
    ((3000, 1000), 2, False, "lorenz_rk4_x2u_kernel<false, 1, true>", True),
    ((3000, 1001), 4, False, "lorenz_rk4_x2u_kernel<false, 2, true>", True),   # ragged total: padded tail
    ((3001, 1000), 4, False, "lorenz_rk4_x2_kernel<false, 2>", False),          # group start not a multiple of 4
    ((3000, 1000), 2, True, "lorenz_rk4_kahan_x2u_kernel", False),
    ((3000, 1000), 1, False, "integrate_kernel<ff::Lorenz, 0, false, false, 1", False),
])
def test_last_launch_reports_the_kernel(counts, ppt, kahan, expect, fused):
    """ff_last_launch names the integrator kernel the dispatch chose and whether the splat
    ran inside it, so callers need not re-derive the library's dispatch rules."""
    groups = [G(c, *LZ_BOX, 1 if t == 0 else -1, 300 + t) for t, c in enumerate(counts)]
    s = make_system("lorenz", LORENZ_PARAMS, groups, 3, ppt=ppt, kahan=kahan)
    view = FUSE_VIEWS["xz"]
    img = torch.zeros((view["height"], view["width"]), dtype=torch.int32, device="cuda")
    s.step_splat(50, 0.001, view, img)
    rec = s.last_launch()
    assert expect in rec["kernel"], rec
    assert rec["fused_splat"] == fused and rec["integrator_launches"] == 1
    assert rec["splat_launches"] == (0 if fused else 1)
    assert rec["grid"] >= 1 and rec["block"] % 32 == 0
    s.set_launch(ppt, 0, 0, 7)  # at most 7 steps per launch: 50 steps are 8 launches
    s.step_splat(50, 0.001, view, img)
    rec = s.last_launch()
    assert rec["integrator_launches"] == 8 and rec["fused_splat"] == fused
    s.step(0, 0.001)  # launches nothing, keeps the record
    assert s.last_launch()["integrator_launches"] == 8
    s.step(10, 0.001)
    rec = s.last_launch()
    assert rec["integrator_launches"] == 2 and not rec["fused_splat"] and rec["splat_launches"] == 0


def test_last_launch_hh3_and_wilson_cowan():
    for rhs, params, dim, box, name in (("hh3", hh3_params(), 15, CASES["hh3"][3], "ff::HH3"),
                                        ("wilson_cowan", WC_PARAMS, 2, ([0, 0], [1, 1]), "ff::WilsonCowan")):
        s = make_system(rhs, params, [G(1000, *box, 1, 5)], dim)
        assert s.last_launch()["kernel"] == ""  # nothing launched yet
        s.step(5, 0.01)
        rec = s.last_launch()
        assert "integrate_kernel<" + name in rec["kernel"], rec
        assert rec["integrator_launches"] == 1 and not rec["fused_splat"]


def test_step_splat_fallbacks_wc_and_host_image():
    groups = [G(999, [0, 0], [1, 1], 1, 3), G(1000, [0, 0], [1, 1], -1, 4)]
    a = make_system("wilson_cowan", WC_PARAMS, groups, 2)
    b = make_system("wilson_cowan", WC_PARAMS, groups, 2)
    view = dict(ndim_view=2, axes=(0, 1), lo=(0.0, 0.0), hi=(1.0, 1.0), width=64, height=64)
    ha = np.zeros((64, 64), np.uint32)
    a.step_splat(50, 0.01, view, ha)  # host image: separate calls inside
    b.step(50, 0.01)
    hb = np.zeros((64, 64), np.uint32)
    b.project_splat(view, hb)
    np.testing.assert_array_equal(get_state(a), get_state(b))
    np.testing.assert_array_equal(ha, hb)
    with pytest.raises(ff.FFError):
        a.step_splat(1, 0.01, dict(view, ndim_view=5), ha)


def test_pipe_rates_are_consistent():
    """ff_pipe_rate, the denominators of the ALU rooflines: the packed FMA does not widen the
    FP32 pipe (FFMA2 lane rate within 15% of FFMA's), no rate exceeds its unit count at the
    maximum clock, and the logistic chain (one ex2 and one rcp per step) runs at the rate of
    two operations sharing one unit, 2 / (1/ex2 + 1/rcp), within 10% -- the model the
    multi-function rooflines use."""
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    r = {name: ff.ff_pipe_rate(op, 0) for name, op in (("ffma", ff.FF_PIPE_FFMA), ("ffma2", ff.FF_PIPE_FFMA2),
                                                      ("ex2", ff.FF_PIPE_EX2), ("rcp", ff.FF_PIPE_RCP),
                                                      ("logistic", ff.FF_PIPE_LOGISTIC))}
    clock = 2.2e9  # above the maximum SM clock of this part
    assert 0.85 <= r["ffma2"] / r["ffma"] <= 1.15
    assert r["ffma"] <= sms * 128 * clock and r["ffma2"] <= sms * 128 * clock
    assert r["ex2"] <= sms * 32 * clock and r["rcp"] <= sms * 32 * clock
    model = 2.0 / (1.0 / r["ex2"] + 1.0 / r["rcp"])
    assert abs(r["logistic"] / model - 1.0) <= 0.10, (r, model)
