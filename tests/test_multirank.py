"""Multi-rank paths on CPU (gloo, world size 2).

Particles are independent, so N GPUs run N weak-scaling shards of a workload with
rank-distinct seeds and no data-path collective; the only cross-rank operation is
the bench harness's max-over-ranks timing.  These tests check, without a GPU, that
shards draw disjoint initial conditions, that the timing reduction returns the
maximum on every rank, and that the reference arm keeps the launch contract under
torch.distributed.run (rank 0 prints one JSON line, the other rank exits 0 quietly).
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_1505_00344_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = W.shard(W.workload("lorenz_4M"), rank, world)
        g = w["groups"][0]
        x = oracle.seed_group(3, g["lo"], g["hi"], g["seed"], count=256)
        xs = [torch.zeros(3, 256) for _ in range(world)]
        dist.all_gather(xs, torch.from_numpy(x))
        t = bench.max_over_ranks(10.0 + rank, "cpu")
        out[rank] = (t, [v.numpy().copy() for v in xs], [gg["count"] for gg in w["groups"]])
    finally:
        dist.destroy_process_group()


def test_weak_shards_are_disjoint_and_timing_takes_the_max():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        t, xs, counts = res[r]
        assert t == 10.0 + (world - 1)  # every rank sees the slowest rank's time
        assert counts == [3145728, 1048576]  # weak scaling: every shard is the full workload
        assert not np.array_equal(xs[0], xs[1])  # rank-distinct seeds give different particles
        np.testing.assert_array_equal(xs[r], res[r][1][r])


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["metric"] == "particle-RK4-steps/sec" and d["higher_is_better"] is True


# ---------------------------------------------------------------------------
# One ensemble split across ranks (contiguous particle ranges) and summed back
# ---------------------------------------------------------------------------
def test_split_ranges_cover_the_ensemble_in_order():
    from paper_1505_00344_gb300 import shards

    for total, world, align in ((4_194_304, 8, 4), (4097, 3, 4), (10, 4, 4), (5, 8, 1), (0, 2, 4)):
        ranges = [shards.split_range(total, r, world, align) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == total
        for (a0, b0), (a1, b1) in zip(ranges, ranges[1:]):
            assert b0 == a1 and a0 <= b0
        for a, b in ranges[:-1]:
            assert b % align == 0 or b == total
    counts = [3001, 999, 4]
    got = shards.group_slices(counts, 2000, 4002)
    assert got == [(0, 2000, 1001, 3001), (1, 0, 999, 999), (2, 0, 2, 4)]
    assert shards.group_slices(counts, 3001, 3001) == []
    assert shards.local_group_mask(0b101, [1, 2]) == 0b10
    assert shards.local_group_mask(0b011, [0, 1, 2]) == 0b011


SPLIT_W = dict(dim=3, params=[10.0, 28.0, 8.0 / 3.0], dt=0.001, steps=150,
               groups=[dict(count=1501, direction=1, seed=77, lo=[-30.0, -30.0, 0.0], hi=[30.0, 30.0, 60.0]),
                       dict(count=503, direction=-1, seed=78, lo=[-30.0, -30.0, 0.0], hi=[30.0, 30.0, 60.0])],
               view=dict(lo=(-30.0, 0.0), hi=(30.0, 60.0), width=64, height=48))


def _oracle_part(w, a, b):
    """Initial states and signed steps of ensemble particles [a, b), from the oracle's seeding."""
    import oracle
    from paper_1505_00344_gb300 import shards

    xs, hs = [], []
    for gi, first, count, _ in shards.group_slices([g["count"] for g in w["groups"]], a, b):
        g = w["groups"][gi]
        xs.append(oracle.seed_group(w["dim"], g["lo"], g["hi"], g["seed"], count=count, j0=first))
        hs.append(np.full(count, g["direction"] * w["dt"]))
    return np.concatenate(xs, axis=1), np.concatenate(hs)


def _oracle_image_and_grad(w, a, b, P):
    """Count image of the particles [a, b) after the run, and their contribution to the
    gradients of L = (1/P) sum_i |x_i(T) - t_i|^2 (targets seeded per ensemble index)."""
    import oracle

    x0, h = _oracle_part(w, a, b)
    xT, S, Q = oracle.tangent(oracle.LORENZ, x0, w["params"], h, w["steps"])
    v = w["view"]
    xf = xT.astype(np.float32)
    img = oracle.splat2d(xf[0], xf[2], v["lo"], v["hi"], v["width"], v["height"])
    tgt = np.random.default_rng(5).uniform(-20.0, 20.0, (w["dim"], P))[:, a:b]
    g = (2.0 / P) * (xT - tgt)
    return img, np.einsum("pij,ip->jp", S, g), np.einsum("piq,ip->q", Q, g)


def _split_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_1505_00344_gb300 import shards

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        P = sum(g["count"] for g in SPLIT_W["groups"])
        a, b = shards.split_range(P, rank, world)
        img, dx0, dp = _oracle_image_and_grad(SPLIT_W, a, b, P)
        image = shards.allreduce_sum(torch.from_numpy(img.view(np.int32).copy()))
        grad = shards.allreduce_sum(torch.from_numpy(dp.copy()))
        out[rank] = (a, b, image.numpy().view(np.uint32).copy(), grad.numpy().copy(), dx0)
    finally:
        dist.destroy_process_group()


def test_split_ensemble_reduces_to_the_single_rank_result():
    """Two gloo ranks each take a contiguous half of one Lorenz ensemble (a forward and a
    backward group, the split falling inside the first), run it in the oracle and sum
    their images and FP64 parameter gradients with shards.allreduce_sum: the image equals
    the one-rank image bit for bit, dL/dp agrees to FP64 summation order and each rank's
    dL/dx0 is the one-rank result for its particles."""
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_split_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = dict(out)
    P = sum(g["count"] for g in SPLIT_W["groups"])
    img, dx0, dp = _oracle_image_and_grad(SPLIT_W, 0, P, P)
    assert res[0][1] == res[1][0] and 0 < res[0][1] < SPLIT_W["groups"][0]["count"]
    for r in range(world):
        a, b, image, grad, dx0_r = res[r]
        np.testing.assert_array_equal(image, img)
        np.testing.assert_allclose(grad, dp, rtol=1e-12, atol=1e-15 * np.abs(dp).max())
        np.testing.assert_array_equal(dx0_r, dx0[:, a:b])
    assert img.sum() > 0
