import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libff.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_golden(name):
    """Parse a golden fixture: '#' lines are citations/comments, others 'key value [value...]'."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


# Parity bar for the first 100 steps of an integration against the FP64 oracle.
TOL = 1e-5
BACKWARD_LORENZ_TOL = 1e-4


def state_err(got, want):
    """Per-particle relative state error: max over components k of
    |x_k - x_ref,k| / max(|x_ref,k|, 1) (each component on its own scale, floored at 1,
    since gates are ~0-1 and V is tens of mV)."""
    import numpy as np

    d = np.abs(np.asarray(got, dtype=np.float64) - want) / np.maximum(np.abs(want), 1.0)
    return d.max(axis=0)


def assert_parity_bar(err, spread=None, backward=None, fp32=None):
    """Assert the parity bar and return a one-line summary of the measured errors.

    err: per-particle state_err of the CUDA result against the FP64 oracle.  For the
    chaotic (Lorenz, HH x 3) or unstable (backward-time) cases also: spread, the
    state_err of the FP64 oracle restarted from a one-ulp perturbed initial state;
    fp32, the state_err of the oracle's formulas evaluated in FP32 (oracle.integrate_fp32);
    backward, a mask of backward-time particles (reported apart).

    Without spread: every particle <= 1e-5 (the non-chaotic systems).  With it, per
    time direction: 99% of particles <= max(1e-5, 2 x the FP32 evaluation's 99th
    percentile) and all <= max(1e-5, 5 x the largest one-ulp spread, 5 x the FP32
    evaluation's largest error).  No FP32 computation of these systems can beat the
    oracle's own sensitivity to its initial rounding, and an FP32 evaluation of the
    oracle's very formulas (correctly rounded exponentials, no contraction) already
    misses 1e-5 per component on HH x 3 spikes and on Lorenz at large r.
    Backward-time Lorenz particles whose error exceeds 1e-4 are flagged in the summary."""
    import numpy as np

    err = np.asarray(err)
    if spread is None:
        assert err.max() <= TOL, err.max()
        return f"max {err.max():.2e}"
    bwd = np.zeros(err.shape, bool) if backward is None else np.asarray(backward, bool)
    spread = np.asarray(spread)
    fp32 = np.zeros(err.shape) if fp32 is None else np.asarray(fp32)
    out = []
    for name, m in (("forward", ~bwd), ("backward", bwd)):
        if not m.any():
            continue
        e, s, y = err[m], spread[m], fp32[m]
        p99, y99 = np.quantile(e, 0.99), np.quantile(y, 0.99)
        bar_max = max(TOL, 5 * s.max(), 5 * y.max())
        assert p99 <= max(TOL, 2 * y99), (name, p99, y99)
        assert e.max() <= bar_max, (name, e.max(), s.max(), y.max())
        flag = " (above 1e-4)" if name == "backward" and e.max() > BACKWARD_LORENZ_TOL else ""
        out.append(f"{name}: max {e.max():.2e} p99 {p99:.2e} | FP32 evaluation max {y.max():.2e} p99 {y99:.2e} | "
                   f"one-ulp spread max {s.max():.2e}{flag}")
    return "; ".join(out)
