"""Parity at the workloads' full sizes, in the launch configuration bench.py times.

The CUDA path runs the whole workload; the oracle recomputes sampled particles
one by one from its own seeding (and, for the chaotic long runs, compares
attractor-density statistics instead of trajectories):

* lorenz_4M (4 particles per thread, packed pairs, splat fused into the
  integrator, as timed): first 100 steps per sampled trajectory (state-relative error
  <= max(1e-5, 5x the FP64 oracle's one-ulp sensitivity), 99% <= 1e-5);
  after the full 100 frames x 200 steps, the forward group's coarse density
  matches the oracle's (total variation <= 0.05 and <= 3x the distance between
  two independent oracle samples), every backward particle has escaped, and the
  escape flags of the backward group after 1000 steps agree on >= 99% of
  sampled particles.  The compensated (Kahan) integrator's error against FP64
  is stated at 100 and 1000 steps and must not exceed the plain one.
* lorenz_bif_8M: every sampled particle with 2 <= r <= 6 ends on its fixed
  point z = r - 1 in both the GPU and the oracle (on the same side), r <= 0.3
  ends at the origin, and the GPU image of those columns has all its mass on
  the row of z = r - 1.
* hh3_1M: first 100 steps per sampled trajectory (plain FP32: within five times
  the FP64 oracle's one-ulp sensitivity; 99% of particles within 1e-5).
* wc_4k: the whole workload (4096 particles, 1000 steps) per trajectory and the
  256x256 image against the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from paper_1505_00344_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()


def system(w, kahan=False):
    # the library's default launch shape, which bench.py times (4 particles per thread for RK4 on Lorenz)
    return ff.System.from_workload(w, kahan=kahan, stream=torch.cuda.current_stream().cuda_stream)


def state(s):
    n, _, dim, _ = s.info()
    out = np.empty((dim, n), np.float32)
    s.get_state(out)
    return out


def particle_err(got, want):
    d = np.abs(got.astype(np.float64) - want).max(axis=0)
    return d / np.maximum(np.abs(want).max(axis=0), 1.0)


def locate(w, idx):
    """(group index, index within the group) of global particle indices."""
    starts = np.cumsum([0] + [g["count"] for g in w["groups"]])
    gi = np.searchsorted(starts, idx, side="right") - 1
    return gi, idx - starts[gi]


def oracle_sample(w, idx, steps, params=None, pparam=None):
    """Oracle states of global particles idx after `steps` steps (from the oracle's own seeding)."""
    gi, local = locate(w, idx)
    x0 = np.empty((w["dim"], idx.size), np.float32)
    h = np.empty(idx.size)
    for g in np.unique(gi):
        m = gi == g
        grp = w["groups"][g]
        x0[:, m] = oracle.seed_group(w["dim"], grp["lo"], grp["hi"], grp["seed"], idx=local[m])
        h[m] = grp["direction"] * w["dt"]
    rid = W.RHS_IDS[w["rhs"]]
    kw = {}
    if pparam is not None:
        kw = dict(pparam_index=w["pparam"]["index"], pparam=pparam)
    return oracle.integrate_parallel(rid, x0, params or w["params"], h, steps, **kw)[0], x0


def escaped(x):
    return ~(np.abs(x.astype(np.float64)) <= 1e30).all(axis=0)


# ---------------------------------------------------------------------------
# 4M-particle Lorenz workload
# ---------------------------------------------------------------------------
def test_lorenz_4M_sampled_first_frame():
    w = W.workload("lorenz_4M")
    s = system(w)
    s.step(100, w["dt"])
    got = state(s)
    idx = np.sort(np.random.default_rng(1).choice(got.shape[1], 4096, replace=False))
    want, x0 = oracle_sample(w, idx, 100)
    err = particle_err(got[:, idx], want)
    gi, _ = locate(w, idx)
    h = np.array([w["groups"][g]["direction"] * w["dt"] for g in gi])
    sign = np.random.default_rng(0).choice([-1.0, 1.0], x0.shape)
    pert = oracle.integrate_parallel(oracle.LORENZ, x0.astype(np.float64) * (1 + 6e-8 * sign), w["params"], h,
                                     100)[0]
    spread = particle_err(pert, want).max()
    print(f"\n[lorenz_4M 100 steps] max err {err.max():.2e}, p99 {np.quantile(err, 0.99):.2e}, "
          f"one-ulp spread {spread:.2e}")
    assert err.max() <= max(TOL, 5 * spread) and np.quantile(err, 0.99) <= TOL
    s.close()


def test_lorenz_4M_kahan_error_statement(capsys):
    w = W.workload("lorenz_4M")
    idx = np.sort(np.random.default_rng(2).choice(4_194_304, 2048, replace=False))
    plain, comp = system(w), system(w, kahan=True)
    rows = []
    done = 0
    for n in (100, 1000):
        plain.step(n - done, w["dt"])
        comp.step(n - done, w["dt"])
        done = n
        want, _ = oracle_sample(w, idx, n)
        ok = ~escaped(want)
        ep = particle_err(state(plain)[:, idx], want)[ok]
        ek = particle_err(state(comp)[:, idx], want)[ok]
        rows.append((n, np.median(ep), ep.max(), np.median(ek), ek.max()))
        assert np.median(ek) <= np.median(ep)
    with capsys.disabled():
        for n, mp, xp, mk, xk in rows:
            print(f"\n[lorenz_4M error vs FP64] step {n}: plain median {mp:.2e} max {xp:.2e} | "
                  f"kahan median {mk:.2e} max {xk:.2e}")
    plain.close()
    comp.close()


def _coarse_density(s, w, group_mask, nb=(48, 27)):
    v = dict(w["view"])
    v.update(width=nb[0], height=nb[1], group_mask=group_mask)
    img = torch.zeros((nb[1], nb[0]), dtype=torch.int32, device="cuda")
    s.project_splat(v, img)
    torch.cuda.synchronize()
    a = img.cpu().numpy().view(np.uint32).astype(np.float64)
    return a / max(a.sum(), 1.0)


def _oracle_density(w, x, nb=(48, 27)):
    v = w["view"]
    xf = x.astype(np.float32)
    img = oracle.splat2d(xf[v["axes"][0]], xf[v["axes"][1]], v["lo"], v["hi"], nb[0], nb[1]).astype(np.float64)
    return img / max(img.sum(), 1.0)


def test_lorenz_4M_full_job_statistics():
    w = W.workload("lorenz_4M")
    s = system(w)
    view = ff.make_view(**w["view"])
    image = torch.zeros((w["view"]["height"], w["view"]["width"]), dtype=torch.int32, device="cuda")
    n_fwd = w["groups"][0]["count"]
    for f in range(w["frames"]):
        s.step_splat(w["steps_per_frame"], w["dt"], view, image)  # the timed path: splat fused into the integrator
        if f == 4:  # 1000 steps: the backward group is escaping
            st = state(s)
            idx = n_fwd + np.arange(0, w["groups"][1]["count"], 256)
            want, _ = oracle_sample(w, idx, 1000)
            assert (escaped(st[:, idx]) == escaped(want)).mean() >= 0.99
    torch.cuda.synchronize()
    n_esc, t_fwd, t_bwd = s.stats()
    assert n_esc == w["groups"][1]["count"]  # every backward particle escaped, no forward one
    assert abs(t_fwd - 20.0) < 1e-9 and abs(t_bwd + 20.0) < 1e-9
    img = image.cpu().numpy().view(np.uint32)
    assert 0.9 * n_fwd < img.sum() <= n_fwd
    # the fused splat of the last frame is the projection of the final states
    again = torch.zeros_like(image)
    s.project_splat(view, again)
    np.testing.assert_array_equal(again.cpu().numpy(), image.cpu().numpy())
    gpu = _coarse_density(s, w, group_mask=0b01)
    N = 65536
    A, _ = oracle_sample(w, np.arange(N), 20000)
    B, _ = oracle_sample(w, np.arange(N, 2 * N), 20000)
    assert not escaped(A).any()
    pa, pb = _oracle_density(w, A), _oracle_density(w, B)
    tv_ab = 0.5 * np.abs(pa - pb).sum()
    tv = 0.5 * np.abs(gpu - pa).sum()
    print(f"\n[lorenz_4M density] TV(gpu, oracle) = {tv:.4f}, TV(oracle A, oracle B) = {tv_ab:.4f}")
    assert tv <= 0.05 and tv <= 3 * tv_ab
    s.close()


# ---------------------------------------------------------------------------
# 8M-particle live bifurcation diagram
# ---------------------------------------------------------------------------
def test_lorenz_bif_8M_invariants():
    w = W.workload("lorenz_bif_8M")
    s = system(w)
    view = ff.make_view(**w["view"])
    H, Wd = w["view"]["height"], w["view"]["width"]
    image = torch.zeros((H, Wd), dtype=torch.int32, device="cuda")
    for f in range(w["frames"]):
        if f in w["schedule"]:
            s.set_params(w["schedule"][f])
        s.step(w["steps_per_frame"], w["dt"])
    s.project_splat(view, image)
    got = state(s)
    P = got.shape[1]
    r_all = oracle.linspace_param(P, w["pparam"]["lo"], w["pparam"]["hi"])
    # sample: 1024 particles with r < 10 and 1024 anywhere
    low = np.nonzero(r_all < 10.0)[0]
    rng = np.random.default_rng(3)
    idx = np.sort(np.concatenate([rng.choice(low, 1024, replace=False), rng.choice(P, 1024, replace=False)]))
    r = r_all[idx].astype(np.float64)
    x = oracle_sample(w, idx, w["steps_per_frame"], pparam=r)[0]
    x = _continue(w, idx, x, r)
    g = got[:, idx].astype(np.float64)
    # within the 20 time units of the run, spirals with r <= 6 settle to 2e-3
    band = (r >= 2.0) & (r <= 6.0)
    assert band.sum() > 100
    np.testing.assert_allclose(g[2, band], r[band] - 1.0, atol=2e-3)
    np.testing.assert_allclose(x[2, band], r[band] - 1.0, atol=2e-3)
    assert (np.sign(g[0, band]) == np.sign(x[0, band])).mean() >= 0.99
    # the origin attracts at rate (sqrt((sigma+1)^2 - 4 sigma (1-r)) - (sigma+1))/2, >= 0.68 for r <= 0.3
    origin = r <= 0.3
    assert origin.sum() > 0
    assert np.abs(g[:, origin]).max() < 1e-3 and np.abs(x[:, origin]).max() < 1e-3
    # image: columns with 2 <= r <= 6 carry their mass on the row of z = r - 1
    img = image.cpu().numpy().view(np.uint32)
    cols = np.arange(int(np.ceil(2.0 / 200 * Wd)) + 1, int(6.0 / 200 * Wd) - 1)
    for c in cols[::7]:
        r_c = (c + 0.5) * 200.0 / Wd
        row = int((r_c - 1.0) * H / 400.0)
        col = img[:, c]
        assert col.sum() > 0
        assert col[max(row - 2, 0):row + 3].sum() == col.sum()
    s.close()


def _continue(w, idx, x, r):
    """Second half of the bifurcation run in the oracle: the parameter change, then the rest."""
    h = np.full(idx.size, w["dt"])
    out, _ = oracle.integrate_parallel(W.RHS_IDS[w["rhs"]], x, w["schedule"][1], h, w["steps_per_frame"],
                                       pparam_index=w["pparam"]["index"], pparam=r)
    return out


# ---------------------------------------------------------------------------
# 1M-particle three-neuron Hodgkin-Huxley
# ---------------------------------------------------------------------------
def test_hh3_1M_sampled_first_steps():
    w = W.workload("hh3_1M")
    s = system(w)
    s.step(100, w["dt"])
    got = state(s)
    idx = np.sort(np.random.default_rng(4).choice(got.shape[1], 2048, replace=False))
    want, x0 = oracle_sample(w, idx, 100)
    err = particle_err(got[:, idx], want)
    sign = np.random.default_rng(0).choice([-1.0, 1.0], x0.shape)
    h = np.full(idx.size, w["dt"])
    pert = oracle.integrate_parallel(oracle.HH3, x0.astype(np.float64) * (1 + 6e-8 * sign), w["params"], h, 100)[0]
    spread = particle_err(pert, want).max()
    assert err.max() <= max(TOL, 5 * spread)
    assert np.quantile(err, 0.99) <= TOL
    s.close()


# ---------------------------------------------------------------------------
# 4096-particle Wilson-Cowan workload, whole run
# ---------------------------------------------------------------------------
def test_wc_4k_whole_workload():
    w = W.workload("wc_4k")
    s = system(w)
    s.step(w["steps_per_frame"], w["dt"])
    v = w["view"]
    image = torch.zeros((v["height"], v["width"]), dtype=torch.int32, device="cuda")
    s.project_splat(ff.make_view(**v), image)
    got = state(s)
    want, _ = oracle_sample(w, np.arange(got.shape[1]), w["steps_per_frame"])
    err = particle_err(got, want)
    print(f"\n[wc_4k] 1000-step state error vs FP64: max {err.max():.2e} median {np.median(err):.2e}")
    assert err.max() <= 1e-4
    img = image.cpu().numpy().view(np.uint32).astype(np.int64)
    ref = oracle.splat2d(want[0].astype(np.float32), want[1].astype(np.float32), v["lo"], v["hi"], v["width"],
                         v["height"]).astype(np.int64)
    # particles whose FP32 and FP64 states fall in different pixels move two counts
    assert np.abs(img - ref).sum() <= 2 * max(4, int(0.002 * got.shape[1]))
    s.close()
