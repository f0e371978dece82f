"""Parity at the workloads' full sizes, in the launch configuration bench.py times.

The CUDA path runs the whole workload; the oracle recomputes sampled particles
one by one from its own seeding (and, for the chaotic long runs, compares
attractor-density statistics instead of trajectories):

* lorenz_4M (4 particles per thread, packed pairs, splat fused into the
  integrator, as timed): first 100 steps per sampled trajectory (per-component
  relative error |x - x_ref| / max(|x_ref|, 1): forward particles <= max(1e-5, 5x
  the FP64 oracle's one-ulp sensitivity) with 99% <= 1e-5, backward ones <= 1e-4);
  after the full 100 frames x 200 steps, the forward group's coarse density
  matches the oracle's (total variation <= 0.05 and <= 3x the distance between
  two independent oracle samples), every backward particle has escaped, and the
  escape flags of the backward group after 1000 steps agree on >= 99.9% of
  sampled particles.  The compensated (Kahan) integrator's error against FP64
  is stated at 100 and 1000 steps (median not above the plain one) and, after
  the decorrelation of the chaotic trajectories, at 20,000 steps as the same
  coarse-density distance for plain and Kahan.
* lorenz_bif_8M: every sampled particle with 2 <= r <= 6 ends on its fixed
  point z = r - 1 in both the GPU and the oracle (on the same side), r <= 0.3
  ends at the origin, and the GPU image of those columns has all its mass on
  the row of z = r - 1; in the chaotic band r >= 25 the (r, z) density of all
  GPU particles matches two disjoint 65,536-particle oracle samples (same
  total-variation bar).
* hh3_1M: first 100 steps per sampled trajectory (within five times the FP64
  oracle's one-ulp sensitivity; 99% of particles within 1e-5), and after the
  whole 50,000-step run the 64x64 density of the (V1, V2, V3) view against two
  disjoint 8,192-particle oracle samples (same total-variation bar).
* wc_4k: the whole workload (4096 particles, 1000 steps) per trajectory and the
  256x256 image against the oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from conftest import TOL, assert_parity_bar, state_err  # noqa: E402
from paper_1505_00344_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu



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


particle_err = state_err


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


def report(capsys, text):
    """Print a measured statement so that it shows in the test log."""
    with capsys.disabled():
        print("\n" + text)


def escaped(x):
    return ~(np.abs(x.astype(np.float64)) <= 1e30).all(axis=0)


# ---------------------------------------------------------------------------
# 4M-particle Lorenz workload
# ---------------------------------------------------------------------------
def test_lorenz_4M_sampled_first_frame(capsys):
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
    fp32 = oracle.integrate_fp32(oracle.LORENZ, x0, w["params"], h, 100)
    summary = assert_parity_bar(err, particle_err(pert, want), h < 0, particle_err(fp32, want))
    report(capsys, f"[lorenz_4M 100 steps, per-component error vs FP64] {summary}")
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


def test_lorenz_4M_full_job_statistics(capsys):
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
            agree = float((escaped(st[:, idx]) == escaped(want)).mean())
            report(capsys, f"[lorenz_4M backward group, step 1000] escape flags agree on {agree:.4%} of "
                           f"{idx.size} sampled particles ({escaped(want).mean():.1%} escaped in the oracle)")
            assert agree >= 0.999
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
    AB, _ = oracle_sample(w, np.arange(2 * N), 20000)
    A, B = AB[:, :N], AB[:, N:]
    assert not escaped(AB).any()
    pa, pb = _oracle_density(w, A), _oracle_density(w, B)
    tv_ab = 0.5 * np.abs(pa - pb).sum()
    tv = 0.5 * np.abs(gpu - pa).sum()
    assert tv <= 0.05 and tv <= 3 * tv_ab
    plain_final = state(s)[:, :N]
    s.close()
    # Error statement of the compensated integrator at step 20,000 (20 time units): the
    # trajectories have decorrelated from the FP64 ones (largest Lyapunov exponent ~0.9), so
    # the statement is statistical -- the same coarse-density distance, for plain and Kahan.
    comp = system(w, kahan=True)
    for f in range(w["frames"]):
        comp.step(w["steps_per_frame"], w["dt"])
    tv_k = 0.5 * np.abs(_coarse_density(comp, w, group_mask=0b01) - pa).sum()
    ep = particle_err(plain_final, A)
    ek = particle_err(state(comp)[:, :N], A)
    comp.close()
    report(capsys, f"[lorenz_4M error vs FP64] step 20000: TV(plain, oracle) = {tv:.4f}, TV(kahan, oracle) = "
          f"{tv_k:.4f}, TV(oracle A, oracle B) = {tv_ab:.4f}; per-trajectory median plain {np.median(ep):.2e} "
          f"kahan {np.median(ek):.2e} (decorrelated)")
    assert tv_k <= 0.05 and tv_k <= 3 * tv_ab


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


def test_lorenz_bif_8M_chaotic_band_density(capsys):
    """Beyond the Hopf point (r > 24.74 at beta = 8/3, 21.4 at beta = 2) most columns of the
    diagram are chaotic: there the (r, z) density of the GPU run over every particle with
    r >= 25 is compared with two disjoint random samples of 65,536 such particles run by
    the oracle (r in 35 bins of 5, z in 20 bins of 20 over [0, 400])."""
    w = W.workload("lorenz_bif_8M")
    s = system(w)
    for f in range(w["frames"]):
        if f in w["schedule"]:
            s.set_params(w["schedule"][f])
        s.step(w["steps_per_frame"], w["dt"])
    nb = (35, 20)
    lo, hi = (25.0, 0.0), (200.0, 400.0)
    v = dict(w["view"], lo=lo, hi=hi, width=nb[0], height=nb[1])
    img = torch.zeros((nb[1], nb[0]), dtype=torch.int32, device="cuda")
    s.project_splat(v, img)
    torch.cuda.synchronize()
    gpu = img.cpu().numpy().view(np.uint32).astype(np.float64)
    P = w["groups"][0]["count"]
    n_esc = s.stats()[0]
    s.close()
    r_all = oracle.linspace_param(P, w["pparam"]["lo"], w["pparam"]["hi"])
    band = np.nonzero(r_all >= 25.0)[0]
    assert n_esc == 0 and gpu.sum() >= band.size - 1  # every band particle drawn but r = 200 (right edge)
    rng = np.random.default_rng(11)
    N = 65536
    idx = np.sort(rng.choice(band, 2 * N, replace=False))
    r = r_all[idx].astype(np.float64)
    x = oracle_sample(w, idx, w["steps_per_frame"], pparam=r)[0]
    x = _continue(w, idx, x, r)
    assert not escaped(x).any()
    perm = rng.permutation(2 * N)

    def dens(sel):
        a = oracle.splat2d(r[sel].astype(np.float32), x[2, sel].astype(np.float32), lo, hi, nb[0], nb[1])
        return a.astype(np.float64) / a.sum()

    pa, pb = dens(perm[:N]), dens(perm[N:])
    gpu /= gpu.sum()
    tv_ab = 0.5 * np.abs(pa - pb).sum()
    tv = 0.5 * np.abs(gpu - pa).sum()
    report(capsys, f"[lorenz_bif_8M chaotic band r >= 25] TV(gpu, oracle) = {tv:.4f}, "
          f"TV(oracle A, oracle B) = {tv_ab:.4f}")
    assert tv <= 0.05 and tv <= 3 * tv_ab


# ---------------------------------------------------------------------------
# 1M-particle three-neuron Hodgkin-Huxley
# ---------------------------------------------------------------------------
def test_hh3_1M_full_run_density(capsys):
    """The whole hh3_1M run (50,000 RK4 steps, 500 ms) in the bench's launch shape, then the
    (V1, V2, V3) view through the workload's camera into a 64 x 64 grid: the GPU density of
    all 1,048,576 particles against two disjoint oracle samples of 8,192 particles
    (Sec. 3, Eq. 6-11; the projection of Fig. 6)."""
    w = W.workload("hh3_1M")
    s = system(w)
    s.step(w["steps_per_frame"], w["dt"])
    nb = 64
    v = dict(w["view"], width=nb, height=nb)
    img = torch.zeros((nb, nb), dtype=torch.int32, device="cuda")
    s.project_splat(v, img)
    torch.cuda.synchronize()
    gpu = img.cpu().numpy().view(np.uint32).astype(np.float64)
    n_esc = s.stats()[0]
    s.close()
    assert n_esc == 0
    N = 8192
    x, _ = oracle_sample(w, np.arange(2 * N), w["steps_per_frame"])
    assert not escaped(x).any()
    ax, mvp = w["view"]["axes"], w["view"]["mvp"]

    def dens(x):
        xf = x.astype(np.float32)
        a = oracle.splat3d(xf[ax[0]], xf[ax[1]], xf[ax[2]], mvp, nb, nb).astype(np.float64)
        return a / a.sum()

    pa, pb = dens(x[:, :N]), dens(x[:, N:])
    gpu /= gpu.sum()
    tv_ab = 0.5 * np.abs(pa - pb).sum()
    tv = 0.5 * np.abs(gpu - pa).sum()
    report(capsys, f"[hh3_1M density after 50,000 steps] TV(gpu, oracle) = {tv:.4f}, "
          f"TV(oracle A, oracle B) = {tv_ab:.4f}")
    assert tv <= 0.05 and tv <= 3 * tv_ab



def test_hh3_1M_sampled_first_steps(capsys):
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
    fp32 = oracle.integrate_fp32(oracle.HH3, x0, w["params"], h, 100)
    summary = assert_parity_bar(err, particle_err(pert, want), None, particle_err(fp32, want))
    report(capsys, f"[hh3_1M 100 steps, per-component error vs FP64] {summary}")
    s.close()


# ---------------------------------------------------------------------------
# 4096-particle Wilson-Cowan workload, whole run
# ---------------------------------------------------------------------------
def test_wc_4k_whole_workload(capsys):
    w = W.workload("wc_4k")
    s = system(w)
    s.step(w["steps_per_frame"], w["dt"])
    v = w["view"]
    image = torch.zeros((v["height"], v["width"]), dtype=torch.int32, device="cuda")
    s.project_splat(ff.make_view(**v), image)
    got = state(s)
    idx = np.arange(got.shape[1])
    want, x0 = oracle_sample(w, idx, w["steps_per_frame"])
    gi, _ = locate(w, idx)
    h = np.array([w["groups"][g]["direction"] * w["dt"] for g in gi])
    err = particle_err(got, want)
    # forward: the stable attractor keeps errors at their one-step size; backward: the
    # particles leave [0,1]^2 on unstable paths (|E|, |I| up to ~2e4 after 10 time
    # units), so rounding is amplified and the unstable-case yardsticks apply
    assert err[h > 0].max() <= TOL
    sign = np.random.default_rng(0).choice([-1.0, 1.0], x0.shape)
    pert = oracle.integrate_parallel(oracle.WILSON_COWAN, x0.astype(np.float64) * (1 + 6e-8 * sign), w["params"], h,
                                     w["steps_per_frame"])[0]
    fp32 = oracle.integrate_fp32(oracle.WILSON_COWAN, x0, w["params"], h, w["steps_per_frame"])
    bwd = h < 0
    summary = assert_parity_bar(err[bwd], particle_err(pert, want)[bwd], np.ones(bwd.sum(), bool),
                                particle_err(fp32, want)[bwd])
    report(capsys, f"[wc_4k 1000 steps, per-component error vs FP64] forward max {err[h > 0].max():.2e}; {summary}")
    img = image.cpu().numpy().view(np.uint32).astype(np.int64)
    ref = oracle.splat2d(want[0].astype(np.float32), want[1].astype(np.float32), v["lo"], v["hi"], v["width"],
                         v["height"]).astype(np.int64)
    # particles whose FP32 and FP64 states fall in different pixels move two counts
    assert np.abs(img - ref).sum() <= 2 * max(4, int(0.002 * got.shape[1]))
    s.close()
