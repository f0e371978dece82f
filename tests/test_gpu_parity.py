"""GPU-vs-oracle parity of every hot-path step, through the C ABI.

* seeding and the per-particle parameter linspace: bit-exact;
* integration (RK4 / Euler, plain / Kahan, 1-2-4 particles per thread, forward
  and backward groups, per-particle parameters, mid-run parameter changes):
  max relative state error |x - x_ref| / max(|x_ref|, 1) <= 1e-5 over the
  first 100 steps against the FP64 oracle started from the same FP32 initial
  conditions;
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
from paper_1505_00344_gb300.workloads import (HH3_BASE, LORENZ_PARAMS, WC_PARAMS, hh3_params,  # noqa: E402
                                              look_at_perspective, random_states)

pytestmark = pytest.mark.gpu

TOL = 1e-5


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


def rel_err(got, want):
    return float(np.max(np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1.0)))


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


def _run_case(name, method, kahan, ppt, counts=(1000, 37), steps=100):
    rhs, params, dim, (lo, hi), dt = CASES[name]
    groups = [G(c, lo, hi, 1 if t == 0 else -1, 4242 + t) for t, c in enumerate(counts)]
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
    got, want, _ = _run_case(name, method, kahan, ppt=1)
    assert rel_err(got, want) <= TOL


@pytest.mark.parametrize("name", ["lorenz", "wc", "harmonic"])
@pytest.mark.parametrize("ppt", [2, 4])
def test_integrate_parity_vector_width(name, ppt):
    got, want, _ = _run_case(name, "rk4", False, ppt=ppt, counts=(4097, 1, 2, 3))
    assert rel_err(got, want) <= TOL


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


def test_per_particle_param_and_midrun_set_params():
    # bifurcation-diagram shape: r per particle over [0, 200]; beta switched to 2 after 50 steps
    P = 6001
    groups = [G(P, [-20, -20, 0], [20, 20, 40], 1, 77)]
    s = make_system("lorenz", LORENZ_PARAMS, groups, 3)
    s.set_particle_param(1, 0.0, 200.0)
    s.step(50, 0.001)
    s.set_params([10.0, 28.0, 2.0])
    s.step(50, 0.001)
    got = get_state(s)
    r = oracle.linspace_param(P, 0.0, 200.0).astype(np.float64)
    x = oracle.integrate(oracle.LORENZ, oracle_seed(groups, 3), LORENZ_PARAMS, 0.001, 50, pparam_index=1, pparam=r)
    x = oracle.integrate(oracle.LORENZ, x, [10.0, 28.0, 2.0], 0.001, 50, pparam_index=1, pparam=r)
    assert rel_err(got, x) <= TOL
    n, tf, tb = s.stats()
    assert n == 0 and abs(tf - 0.1) < 1e-15 and tb == 0.0


def test_chunked_launches_match_single_launch():
    rhs, params, dim, (lo, hi), dt = CASES["lorenz"]
    groups = [G(3000, lo, hi, 1, 1), G(1000, lo, hi, -1, 2)]
    a = make_system(rhs, params, groups, dim)
    b = make_system(rhs, params, groups, dim)
    b.set_launch(1, 128, 1, 7)
    a.step(100, dt)
    b.step(100, dt)
    np.testing.assert_array_equal(get_state(a), get_state(b))


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
