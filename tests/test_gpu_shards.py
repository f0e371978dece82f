"""One ensemble split across ranks through the CUDA library (shards.py), on one GPU.

Two processes share cuda:0 and each runs its contiguous share of an ensemble with
the library (ff_seed_particles_slice, ff_set_particle_param_slice); none of their
kernels waits on the other.  The per-frame count images and the FP64 parameter
gradients are summed over gloo (CPU tensors), and every rank compares with the
same ensemble run whole in its own process:

* the reduced image of every frame equals the whole ensemble's image bit for bit,
  and each rank's final states are the whole run's states of its particles;
* a per-particle-parameter ensemble (the bifurcation diagram's r linspace, with the
  beta change between frames) reduces to the whole image too;
* the reverse sweep: each rank's dL/dx0 is the whole run's for its particles, and
  the summed dL/dp matches within the order of FP64 additions;
* particles reset in-kernel (age limit) are re-drawn as members of their whole group.

(With NCCL and one GPU per rank the same calls are the multi-GPU path; no run here
uses more than one GPU.)
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1505_00344_gb300 as ff  # noqa: E402
from paper_1505_00344_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _state(s):
    n, _, dim, _ = s.info()
    x = np.empty((dim, n), np.float32)
    s.get_state(x)
    return x


def _frames(s, w, view, frames, image):
    """Run `frames` frames (parameter schedule applied), splatting each into `image`;
    yields after every frame."""
    schedule = {int(k): v for k, v in w.get("schedule", {}).items()}
    for f in range(frames):
        if f in schedule:
            s.set_params(schedule[f])
        s.step_splat(w["steps_per_frame"], w["dt"], view, image)
        yield f


def _worker(rank, world, port, name, particles, frames, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import paper_1505_00344_gb300 as ff
    from paper_1505_00344_gb300 import shards
    from paper_1505_00344_gb300 import workloads as W

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        stream = torch.cuda.current_stream().cuda_stream
        w = W.scaled(W.workload(name), particles)
        w = dict(w, steps_per_frame=min(w["steps_per_frame"], 500))
        P = sum(g["count"] for g in w["groups"])
        view = ff.make_view(**w["view"])
        H, Wd = w["view"]["height"], w["view"]["width"]
        part, groups, (a, b) = shards.shard_system(w, rank, world, stream=stream)
        whole = ff.System.from_workload(w, stream=stream)
        img_part = torch.zeros((H, Wd), dtype=torch.int32, device="cuda")
        img_whole = torch.zeros_like(img_part)
        res = {"range": (a, b), "frames_equal": [], "drawn": 0}
        for _ in zip(_frames(part, w, view, frames, img_part), _frames(whole, w, view, frames, img_whole)):
            torch.cuda.synchronize()
            summed = shards.allreduce_sum(img_part.cpu())
            res["frames_equal"].append(bool(torch.equal(summed, img_whole.cpu())))
            res["drawn"] = int(summed.sum())
        # (escaped backward particles are NaN in both: compared as equal)
        res["states_equal"] = bool(np.array_equal(_state(part), _state(whole)[:, a:b], equal_nan=True))
        res["launch"] = part.last_launch()["kernel"]
        if name == "lorenz_4M":
            # reverse sweep: L = (1/P) sum |x(T) - t|^2, each rank its particles' share
            n, K = 300, 100
            gen = torch.Generator().manual_seed(11)
            tgt = torch.empty((3, P)).uniform_(-20.0, 20.0, generator=gen).cuda()
            grads = {}
            for key, s, lo, hi in (("part", part, a, b), ("whole", whole, 0, P)):
                s.reset()
                s.tape_begin(K, n)
                s.step(n, w["dt"])
                x = torch.empty((3, hi - lo), dtype=torch.float32, device="cuda")
                s.get_state(x)
                g = (x - tgt[:, lo:hi]) * (2.0 / P)
                dx0 = torch.empty_like(g)
                dp = s.backward(g.contiguous(), dx0, len(w["params"]))
                grads[key] = (dx0.cpu().numpy(), torch.from_numpy(np.array(dp, np.float64)))
                s.tape_end()
            dp_sum = shards.allreduce_sum(grads["part"][1].clone()).numpy()
            dp_whole = grads["whole"][1].numpy()
            res["dx0_equal"] = bool(np.array_equal(grads["part"][0], grads["whole"][0][:, a:b]))
            res["dp_rel"] = float(np.max(np.abs(dp_sum - dp_whole) / np.maximum(np.abs(dp_whole), 1e-300)))
            res["dp_whole"] = dp_whole.tolist()
            # in-kernel reset by age: a shard re-draws its particles as members of the whole group
            for s in (part, whole):
                s.reset()
                s.set_reset(None, None, t_max=30 * w["dt"], check_every=1)
                s.step(100, w["dt"])
            xp, xw = _state(part), _state(whole)[:, a:b]
            res["reset_equal"] = bool(np.array_equal(xp, xw, equal_nan=True))
        out[rank] = res
        part.close()
        whole.close()
    finally:
        dist.destroy_process_group()


def _run(name, particles, frames, world=2):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, name, particles, frames, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=600)
            assert p.exitcode == 0
        return dict(out)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ff.lib()


def test_split_lorenz_images_states_and_gradients():
    res = _run("lorenz_4M", 262_144, 3)
    assert res[0]["range"][1] == res[1]["range"][0]
    # the split falls inside the forward group, on a multiple of 4: both shards keep the fused kernel
    assert 0 < res[0]["range"][1] < 196_608
    for r in (0, 1):
        assert all(res[r]["frames_equal"]) and len(res[r]["frames_equal"]) == 3
        flags = {k: res[r][k] for k in ("states_equal", "dx0_equal", "reset_equal")}
        assert all(flags.values()), (r, flags)
        assert "lorenz_rk4_x2u_kernel<false, 2, true>" in res[r]["launch"]
        # dL/dp: the same FP32 per-particle contributions, summed in FP64 in another order
        assert res[r]["dp_rel"] <= 1e-9, res[r]["dp_rel"]
    assert res[0]["drawn"] > 0


def test_split_bifurcation_diagram_with_parameter_slices():
    res = _run("lorenz_bif_8M", 131_072, 2)
    for r in (0, 1):
        assert all(res[r]["frames_equal"]) and res[r]["states_equal"]
    assert res[0]["drawn"] > 0
