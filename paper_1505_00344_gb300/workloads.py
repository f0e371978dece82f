"""Seeded synthetic workloads shared by the tests, the bench and the CPU oracle legs.

This module holds the *inputs* only: system constants, particle-group boxes,
seeds, step sizes, views and camera matrices, plus seeded random state
generators for tests of the projection step.  It contains none of the method's
arithmetic (no right-hand side, no integrator, no projection), so both the
CUDA path and the FP64 oracle can take their inputs from here without sharing
any computation.

The five workloads follow the paper's example systems:
  * ``wc_4k``        -- Wilson-Cowan E-I model (Eq. 1-2), 4096 particles, half
                        forward / half backward in time, 256x256 view.
  * ``lorenz_4M``    -- Lorenz (Eq. 3-5), 4,194,304 particles, 75% forward /
                        25% backward, 100 frames of 200 RK4 steps, x-z view
                        1920x1080 (the throughput workload).
  * ``lorenz_bif_8M``-- Lorenz live bifurcation diagram (Sec. 2.2, Fig. 4):
                        8,388,608 particles each with its own r, (r, z) view
                        2048x1024, beta switched to 2 after 10,000 steps.
  * ``hh3_1M``       -- three coupled Hodgkin-Huxley neurons (Eq. 6-11),
                        1,048,576 particles, 50,000 steps, 3D (V1,V2,V3) view.
"""
from __future__ import annotations

import math

import numpy as np

RHS_IDS = {"linear": 0, "harmonic": 1, "wilson_cowan": 2, "lorenz": 3, "hh3": 4}
DIMS = {"harmonic": 2, "wilson_cowan": 2, "lorenz": 3, "hh3": 15}

# Wilson-Cowan parameter order: [wEE, wEI, wIE, wII, P, Q, tauE, tauI, gain, threshold]
WC_PARAMS = [16.0, 12.0, 15.0, 3.0, 1.25, 0.0, 1.0, 1.0, 1.0, 4.0]
# Lorenz parameter order: [sigma, r, beta]
LORENZ_PARAMS = [10.0, 28.0, 8.0 / 3.0]
# Hodgkin-Huxley x3 parameter order:
# [C, gNa, gK, gL, ENa, EK, EL, gsyn, Esyn, I1, I2, I3, tau_r, tau_d, sig, theta]
HH3_BASE = [1.0, 120.0, 36.0, 0.3, 50.0, -77.0, -54.4, 0.5, -80.0, 10.0, 10.0, 10.0,
            0.1, 10.0, 0.5, -20.0]

BASE_SEED = 1234


def group_seed(config_index: int, group_index: int) -> int:
    """Seed of one particle group: 1234 + config index, groups spaced by 0x100."""
    return BASE_SEED + config_index + 0x100 * group_index


def hh3_params(seed: int = BASE_SEED + 3):
    """HH3 constants with drive currents I_1..I_3 drawn uniform in [5, 15] uA/cm^2."""
    p = list(HH3_BASE)
    rng = np.random.default_rng(seed)
    p[9:12] = [float(v) for v in rng.uniform(5.0, 15.0, 3)]
    return p


def look_at_perspective(eye, target, up, fovy_deg, aspect, near, far):
    """Column-major 4x4 Model-View-Projection matrix of a pinhole camera.

    Standard right-handed look-at view matrix followed by the standard OpenGL
    perspective projection; this is the camera *input* of a 3D view.
    """
    eye = np.asarray(eye, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    up = np.asarray(up, dtype=np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    view = np.eye(4)
    view[0, :3], view[1, :3], view[2, :3] = s, u, -f
    view[:3, 3] = -view[:3, :3] @ eye
    t = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    proj = np.zeros((4, 4))
    proj[0, 0] = t / aspect
    proj[1, 1] = t
    proj[2, 2] = (far + near) / (near - far)
    proj[2, 3] = 2.0 * far * near / (near - far)
    proj[3, 2] = -1.0
    mvp = proj @ view
    return mvp.T.reshape(16).astype(np.float32)  # column-major


def _wc_4k():
    box = dict(lo=[0.0, 0.0], hi=[1.0, 1.0])
    return dict(
        name="wc_4k", index=0, rhs="wilson_cowan", dim=2, params=list(WC_PARAMS), method="rk4",
        groups=[dict(count=2048, direction=+1, seed=group_seed(0, 0), **box),
                dict(count=2048, direction=-1, seed=group_seed(0, 1), **box)],
        dt=0.01, steps_per_frame=1000, frames=1,
        view=dict(ndim_view=2, axes=(0, 1), lo=(0.0, 0.0), hi=(1.0, 1.0), width=256, height=256),
        # the paper's reset region: the unit square of population activities (Sec. 2.1)
        reset=dict(lo=[0.0, 0.0], hi=[1.0, 1.0], t_max=5.0, check_every=1),
    )


def _lorenz_4M():
    box = dict(lo=[-30.0, -30.0, 0.0], hi=[30.0, 30.0, 60.0])
    return dict(
        name="lorenz_4M", index=1, rhs="lorenz", dim=3, params=list(LORENZ_PARAMS), method="rk4",
        groups=[dict(count=3145728, direction=+1, seed=group_seed(1, 0), **box),
                dict(count=1048576, direction=-1, seed=group_seed(1, 1), **box)],
        dt=0.001, steps_per_frame=200, frames=100, splat_every_frame=True,
        view=dict(ndim_view=2, axes=(0, 2), lo=(-30.0, 0.0), hi=(30.0, 60.0), width=1920, height=1080),
        # optional recycling of escaping backward particles (not part of the measured workload)
        reset=dict(lo=[-60.0, -60.0, -20.0], hi=[60.0, 60.0, 100.0], t_max=0.0, check_every=10),
    )


def _lorenz_bif_8M():
    box = dict(lo=[-20.0, -20.0, 0.0], hi=[20.0, 20.0, 40.0])
    return dict(
        name="lorenz_bif_8M", index=2, rhs="lorenz", dim=3, params=list(LORENZ_PARAMS),
        method="rk4",
        groups=[dict(count=8388608, direction=+1, seed=group_seed(2, 0), **box)],
        dt=0.001, steps_per_frame=10000, frames=2,
        pparam=dict(index=1, lo=0.0, hi=200.0),
        # parameter changes applied before the given frame: beta -> 2.0 after 10,000 steps
        schedule={1: [10.0, 28.0, 2.0]},
        # axis 3 (== dim) is the per-particle parameter r
        view=dict(ndim_view=2, axes=(3, 2), lo=(0.0, 0.0), hi=(200.0, 400.0), width=2048, height=1024),
    )


def _hh3_1M():
    lo = []
    hi = []
    for _ in range(3):
        lo += [-80.0, 0.0, 0.0, 0.0, 0.0]
        hi += [40.0, 1.0, 1.0, 1.0, 1.0]
    mvp = look_at_perspective((150.0, 150.0, 150.0), (-20.0, -20.0, -20.0), (0.0, 0.0, 1.0),
                              45.0, 1.0, 1.0, 1000.0)
    return dict(
        name="hh3_1M", index=3, rhs="hh3", dim=15, params=hh3_params(), method="rk4",
        groups=[dict(count=1048576, direction=+1, seed=group_seed(3, 0), lo=lo, hi=hi)],
        dt=0.01, steps_per_frame=50000, frames=1,
        view=dict(ndim_view=3, axes=(0, 5, 10), mvp=mvp, width=1024, height=1024),
    )


def batch_workload(name: str) -> list:
    """Batched workloads: a list of single-system workloads stepped together.

    * ``hh3_batch64``: 64 three-neuron Hodgkin-Huxley systems of 16,384 particles, coupling
      strengths gsyn = linspace(0, 1, 64), each with its own seeded drive currents.
    * ``mixed_batch256``: 256 systems cycling Wilson-Cowan, Lorenz and HH3 (system s has type
      s mod 3) with particle counts drawn log-uniform between 1,024 and 1,048,576 (seeded).
    """
    hh = _hh3_1M()
    if name == "hh3_batch64":
        out = []
        for k, g in enumerate(np.linspace(0.0, 1.0, 64)):
            w = dict(hh, name=f"hh3_batch64_{k}")
            p = hh3_params(BASE_SEED + 3 + 1000 * k)
            p[7] = float(g)
            w["params"] = p
            w["groups"] = [dict(hh["groups"][0], count=16384, seed=group_seed(3, 0) + 7919 * k)]
            out.append(w)
        return out
    if name == "mixed_batch256":
        rng = np.random.default_rng(BASE_SEED + 4)
        sizes = np.rint(np.exp(rng.uniform(np.log(1024), np.log(1048576), 256))).astype(int)
        bases = (_wc_4k(), _lorenz_4M(), hh)
        out = []
        for k, n in enumerate(sizes):
            b = bases[k % 3]
            w = dict(b, name=f"mixed_batch256_{k}")
            if b["rhs"] == "hh3":
                w["params"] = hh3_params(BASE_SEED + 3 + 1000 * k)
            g0 = b["groups"][0]
            w["groups"] = [dict(g0, count=int(n), direction=1, seed=group_seed(4, 0) + 7919 * k)]
            out.append(w)
        return out
    raise KeyError(name)


WORKLOADS = {w["name"]: w for w in (_wc_4k(), _lorenz_4M(), _lorenz_bif_8M(), _hh3_1M())}


def workload(name: str) -> dict:
    """A fresh copy of a named workload description."""
    return {"wc_4k": _wc_4k, "lorenz_4M": _lorenz_4M, "lorenz_bif_8M": _lorenz_bif_8M,
            "hh3_1M": _hh3_1M}[name]()


def scaled(w: dict, particles: int) -> dict:
    """The same workload with its groups' counts scaled to about ``particles`` in total.

    Group proportions, boxes, seeds and directions are kept; every group keeps
    at least one particle.
    """
    w = dict(w)
    total = sum(g["count"] for g in w["groups"])
    groups = []
    for g in w["groups"]:
        g = dict(g)
        g["count"] = max(1, int(round(g["count"] * particles / total)))
        groups.append(g)
    w["groups"] = groups
    return w


def shard(w: dict, rank: int, world: int) -> dict:
    """Weak-scaling shard for one rank: the full workload with rank-distinct group seeds."""
    w = dict(w)
    groups = []
    for g in w["groups"]:
        g = dict(g)
        g["seed"] = g["seed"] + (rank << 32)
        groups.append(g)
    w["groups"] = groups
    return w


def random_states(dim: int, n: int, lo, hi, seed: int, specials: bool = False) -> np.ndarray:
    """Seeded float32 SoA states [dim][n], uniform in the box [lo, hi).

    With ``specials`` a fixed set of entries is replaced by NaN, +-inf, huge
    values and values on the box edges, to exercise the projection's dropping
    rules.
    """
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64).reshape(-1, 1)
    hi = np.asarray(hi, dtype=np.float64).reshape(-1, 1)
    x = (lo + (hi - lo) * rng.random((dim, n))).astype(np.float32)
    if specials and n >= 16:
        cols = rng.choice(n, size=min(n, 64), replace=False)
        vals = np.array([np.nan, np.inf, -np.inf, 1e30, -1e30, 3e38], dtype=np.float32)
        for t, c in enumerate(cols):
            k = t % dim
            if t < 24:
                x[k, c] = vals[t % vals.size]
            elif t < 44:
                x[k, c] = np.float32(lo[k, 0])
            else:
                x[k, c] = np.float32(hi[k, 0])
    return x
