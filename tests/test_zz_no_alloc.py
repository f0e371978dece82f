"""ff_count_escaped_noalloc: per-group escape counts without any device allocation.

Callers that may not allocate device memory when they ask for statistics (a
plugin given device buffers by a host application that owns the memory budget,
a render loop that cannot take cudaMalloc's synchronisation, a fixed memory pool)
use this entry point instead of ff_stats.  Its counts must equal what ff_stats
reports through the allocating path (the total over all groups, and each group on
its own: a system holding only that group's particles) and what the FP64 oracle's
escape count gives for each group.  Two calls in a row with different data check
that the shared fixed scratch is cleared between calls; a state whose planes are
padded (pitch > n_particles, NaN in the padding) checks that only the first
n_particles of each plane are read, and an empty state gives zero counts.

This file is collected last so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
import paper_1505_00344_gb300 as ff  # noqa: E402
from paper_1505_00344_gb300.workloads import LORENZ_PARAMS, random_states  # noqa: E402


def test_noalloc_rejects_bad_arguments_on_host():
    # host-side checks return before any CUDA call, so this runs without a GPU as well
    L = ff.lib()
    counts = np.zeros(300, np.int64)
    starts = np.zeros(300, np.int64)
    p = counts.ctypes.data
    assert L.ff_count_escaped_noalloc(None, 3, 10, 10, starts.ctypes.data, 1, None, p) == ff.FF_ERR_INVALID_ARG
    fake = 1 << 40  # never dereferenced: the arguments are rejected first
    assert L.ff_count_escaped_noalloc(fake, 3, 10, 10, starts.ctypes.data, 257, None, p) == ff.FF_ERR_INVALID_ARG
    assert "FF_NOALLOC_MAX_GROUPS" in ff.ff_last_error()
    assert L.ff_count_escaped_noalloc(fake, 0, 10, 10, starts.ctypes.data, 1, None, p) == ff.FF_ERR_INVALID_ARG
    assert L.ff_count_escaped_noalloc(fake, 3, 10, 5, starts.ctypes.data, 1, None, p) == ff.FF_ERR_INVALID_ARG
    bad = np.array([1, 2], np.int64)
    assert L.ff_count_escaped_noalloc(fake, 3, 10, 10, bad.ctypes.data, 2, None, p) == ff.FF_ERR_INVALID_ARG
    bad = np.array([0, 7, 3], np.int64)
    assert L.ff_count_escaped_noalloc(fake, 3, 10, 10, bad.ctypes.data, 3, None, p) == ff.FF_ERR_INVALID_ARG
    bad = np.array([0, 11], np.int64)
    assert L.ff_count_escaped_noalloc(fake, 3, 10, 10, bad.ctypes.data, 2, None, p) == ff.FF_ERR_INVALID_ARG


def test_noalloc_binding_rejects_wrong_dtype_or_short_tensor():
    # checked in the binding before the library is called, so no GPU is needed
    starts = [0]
    with pytest.raises(ValueError, match="dtype"):
        ff.ff_count_escaped_noalloc(torch.zeros((3, 100), dtype=torch.float64), 3, 100, 100, starts)
    with pytest.raises(ValueError, match="dtype"):
        ff.ff_count_escaped_noalloc(torch.zeros((3, 100), dtype=torch.float16), 3, 100, 100, starts)
    with pytest.raises(ValueError, match="elements"):
        ff.ff_count_escaped_noalloc(torch.zeros(2 * 128 + 99, dtype=torch.float32), 3, 100, 128, starts)
    with pytest.raises(ValueError):
        ff.ff_count_escaped_noalloc(torch.zeros((3, 100), dtype=torch.float32), 3, 100, 50, starts)


def _states(P, seed, frac_nan):
    x = random_states(3, P, [-50, -50, -50], [50, 50, 50], seed=seed, specials=True)
    rng = np.random.default_rng(seed)
    cols = rng.choice(P, int(frac_nan * P), replace=False)
    x[rng.integers(0, 3, cols.size), cols] = np.nan
    return x


def _reference_counts(x, starts, stream):
    """Escaped particles per group through the allocating path (ff_stats)."""
    P = x.shape[1]
    bounds = list(starts) + [P]
    out = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        if b == a:
            out.append(0)
            continue
        with ff.System("lorenz", LORENZ_PARAMS, b - a, stream=stream) as s:
            s.seed(b - a, [0, 0, 0], [1, 1, 1], 1, 1)
            s.set_state(np.ascontiguousarray(x[:, a:b]))
            out.append(s.stats()[0])
    return np.array(out, np.int64)


@pytest.mark.gpu
def test_noalloc_counts_match_ff_stats_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        (200_003, [0, 1, 5000, 5000, 150_000], 0.02, 7),              # ragged groups, one empty
        (65_536, list(range(0, 65_536, 256)), 0.30, 8),               # the maximum of 256 groups
    ]
    for P, starts, frac, seed in cases:
        x = _states(P, seed, frac)
        with ff.System("lorenz", LORENZ_PARAMS, P, stream=stream) as s:
            s.seed(P, [0, 0, 0], [1, 1, 1], 1, 1)
            s.set_state(x)
            total_ref = s.stats()[0]
            dev = torch.empty((3, P), dtype=torch.float32, device="cuda")
            s.get_state(dev)  # device copy of the state, pitch = P
        counts = ff.ff_count_escaped_noalloc(dev, 3, P, P, starts, stream=stream)
        assert counts.dtype == np.int64 and counts.size == len(starts)
        assert counts.sum() == total_ref > 0
        np.testing.assert_array_equal(counts, _reference_counts(x, starts, stream))
        np.testing.assert_array_equal(counts, _oracle_counts(x, starts))


def _oracle_counts(x, starts):
    """Escaped particles per group from the FP64 oracle's escape test."""
    bounds = list(starts) + [x.shape[1]]
    return np.array([oracle.count_escaped(x[:, a:b])[0] if b > a else 0 for a, b in zip(bounds[:-1], bounds[1:])],
                    np.int64)


@pytest.mark.gpu
def test_noalloc_padded_planes_and_empty_state():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    stream = torch.cuda.current_stream().cuda_stream
    P, pad = 10_007, 245
    x = _states(P, 9, 0.05)
    dev = torch.full((3, P + pad), float("nan"), dtype=torch.float32, device="cuda")
    dev[:, :P] = torch.from_numpy(x).cuda()
    starts = [0, 3, 4096, 9000]
    counts = ff.ff_count_escaped_noalloc(dev, 3, P, P + pad, starts, stream=stream)
    np.testing.assert_array_equal(counts, _oracle_counts(x, starts))
    assert counts.sum() < P  # the NaN padding was not read
    # no particles: no launch, the counters still come back cleared
    counts = ff.ff_count_escaped_noalloc(dev, 3, 0, P + pad, [0, 0], stream=stream)
    np.testing.assert_array_equal(counts, np.zeros(2, np.int64))
