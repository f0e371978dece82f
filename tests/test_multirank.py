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
