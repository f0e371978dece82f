"""Throughput bench of the Fireflies hot path on GB300.

One bench step = one whole run of the 4M-particle Lorenz workload: re-seed both
particle groups (3,145,728 forward, 1,048,576 backward in time), then 100 frames
of 200 RK4 steps (dt = 0.001) each followed by the x-z projection and count splat
into a cleared 1920x1080 image.  Metric: particle-RK4-steps per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own shard (the full workload with rank-distinct
seeds: weak scaling, no data-path collective); value = particles of all ranks x
steps / max-over-ranks time.  ``--impl reference`` times the FP64 CPU oracle on
a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1505_00344_gb300 import workloads as W  # noqa: E402

METRIC = "particle-RK4-steps/sec"
UNIT = "particle-steps/s"
# FP32 instructions / flops of one RK4 step of one Lorenz particle, counted from Eq. 3-5 with
# FMA = 2 flops: RHS 6 instructions (8 flops) x 4 stages, 9 stage updates (18 flops), weighted
# sum + update 12 instructions (21 flops).
LORENZ_RK4_FLOPS = 71
KAHAN_EXTRA_FLOPS = 9
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="lorenz_4M")
    # launch shape (default: the library's default for the system)
    ap.add_argument("--ppt", type=int, default=0)
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--kahan", action="store_true")
    ap.add_argument("--reset", action="store_true", help="enable the workload's particle reset (not the default)")
    ap.add_argument("--adjoint", action="store_true",
                    help="time the taped forward and the adjoint (ff_backward) instead of the plain job")
    ap.add_argument("--adjoint-steps", type=int, default=2000)
    ap.add_argument("--batch", default="", help="time a batched workload (hh3_batch64, mixed_batch256)")
    ap.add_argument("--batch-steps", type=int, default=1000)
    ap.add_argument("--checkpoint-every", type=int, default=100)
    ap.add_argument("--sprites", type=float, default=0.0,
                    help="render soft sprites of this radius (pixels) instead of counts, and time them")
    ap.add_argument("--sprite-technique", choices=["auto", "direct", "tiled"], default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the headline workload (no adjoint and per-workload sub-records)")
    # profiling cases only (a line taken with these is not the workload's number)
    ap.add_argument("--particles", type=int, default=0, help="scale the workload to this many particles")
    ap.add_argument("--frames", type=int, default=0, help="run only this many frames per step")
    ap.add_argument("--frame-steps", type=int, default=0, help="RK4 steps per frame (profiling cases)")
    return ap.parse_args()


def workload_for(args, rank, world):
    w = W.shard(W.workload(args.workload), rank, world)
    if args.particles:
        w = W.scaled(w, args.particles)
    if args.frames:
        w = dict(w, frames=args.frames)
    if args.frame_steps:
        w = dict(w, steps_per_frame=args.frame_steps)
    return w


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def max_over_ranks(x, device):
    """Largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def total_particles(w):
    return sum(g["count"] for g in w["groups"])


def total_steps(w):
    return w["steps_per_frame"] * w["frames"]


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, enabled=True):
        self.proc = None
        self.device_index = device_index
        self.path = os.path.join(tempfile.gettempdir(), f"ff_bench_clocks_{os.getpid()}_{device_index}.csv")
        if not enabled:
            return
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def traffic_from_profile(kernel_src_hash):
    """Per-launch DRAM bytes of the integrator from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "integrate_lorenz_4M_ncu.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != kernel_src_hash:
        return None
    return float(m.group(1))


def _between(text, start, end):
    """The part of text from the line holding `start` up to (not including) `end`."""
    i = text.index(start)
    i = text.rfind("\n", 0, i) + 1
    return text[i:text.index(end, i)]


def kernel_source_hash():
    """Hash of the source the fused Lorenz integrator is compiled and launched from: its
    argument block, step loop, vector loads, packed-pair section, group-uniform launch and
    warp-major item order of ff_device.cuh, the view/pixel rule, ff_integrate_lorenz.cu and the
    default launch shape in ff_api.cu.  A profile taken on other
    sources gives no traffic."""
    csrc = os.path.join(ROOT, "paper_1505_00344_gb300", "csrc")
    dev = open(os.path.join(csrc, "ff_device.cuh")).read()
    proj = open(os.path.join(csrc, "ff_project.cuh")).read()
    api = open(os.path.join(csrc, "ff_api.cu")).read()
    parts = [_between(dev, "struct IntegrateArgs {", "\n};\n") ,
             _between(dev, "// Vector access of PPT consecutive floats.", "// Reset test and re-draw"),
             _between(dev, "// Packed-pair RK4 for Lorenz.", "// Host-side launch of one integrator"),
             _between(dev, "// Deal the persistent grid's blocks out to the groups", "inline cudaError_t launch_variants("),
             _between(dev, "// First item of this thread in a grid-stride loop", "// Minimum resident blocks"),
             _between(dev, "// Checkpoint slot for the state as the launch loads it", "// Reset data of a system"),
             _between(api, "const bool packed_lorenz", "*out = s;"),  # default launch shape
             _between(proj, "struct ViewArgs {", "// Continuous pixel coordinates"),
             open(os.path.join(csrc, "ff_integrate_lorenz.cu")).read()]
    h = hashlib.sha256()
    for part in parts:
        h.update(part.encode())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# MUFU operations of one RK4 step, counted from the equations (exp and reciprocal or
# division each one multi-function-unit operation): Wilson-Cowan per right-hand side
# 2 logistic functions = 2 exp + 2 reciprocals, x 4 stages; Hodgkin-Huxley x 3 per neuron
# and right-hand side 7 exp (six rates + the synaptic activation) + 4 divisions, x 3
# neurons x 4 stages.
MUFU_PER_STEP = {"wilson_cowan": (8, 8), "hh3": (84, 48)}  # (exp, reciprocal)


def pipe_rates(device_index):
    """Measured lane-operation rates of the integrators' instruction kinds (ff_pipe_rate)."""
    import paper_1505_00344_gb300 as ff

    r = {"ffma_lane_ops_per_s": ff.ff_pipe_rate(ff.FF_PIPE_FFMA, device_index),
         "ffma2_lane_ops_per_s": ff.ff_pipe_rate(ff.FF_PIPE_FFMA2, device_index),
         "ex2_per_s": ff.ff_pipe_rate(ff.FF_PIPE_EX2, device_index),
         "rcp_per_s": ff.ff_pipe_rate(ff.FF_PIPE_RCP, device_index),
         "logistic_mufu_ops_per_s": ff.ff_pipe_rate(ff.FF_PIPE_LOGISTIC, device_index),
         "how": "ff_pipe_rate: 8 independent chains per thread, full occupancy, 4096 iterations, CUDA events"}
    # ex2 and rcp share the multi-function unit when the logistic chain (one of each) runs at
    # 2 / (1/ex2 + 1/rcp); the MUFU rooflines use that model
    r["shared_unit_model_logistic"] = 2.0 / (1.0 / r["ex2_per_s"] + 1.0 / r["rcp_per_s"])
    return r


def roofline_for(w, n_work, avg_launch_ms, steps_per_launch, sms, max_mhz, rates, kahan=False):
    """ALU roofline of one integrator launch: FP32 flops for Lorenz against the FP32 peak
    derived from unit counts and the clock; multi-function-unit operations for Wilson-Cowan and
    HH x 3 against the measured ex2 / reciprocal rates for their mix."""
    if w["rhs"] == "lorenz":
        step_flops = LORENZ_RK4_FLOPS + (KAHAN_EXTRA_FLOPS if kahan else 0)
        work = step_flops * n_work * steps_per_launch
        achieved = work / (avg_launch_ms / 1e3) / 1e12
        peak = sms * FP32_LANES_PER_SM * 2 * max_mhz * 1e6 / 1e12
        out = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
               "frac": round(achieved / peak, 4),
               "peak_basis": f"FP32 FMA: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 flop x {max_mhz:.0f} MHz "
                             "(max SM clock)",
               "work_per_particle_step": f"{step_flops} flop (Eq. 3-5, FMA = 2 flops)"}
        if rates:
            m = 2 * rates["ffma2_lane_ops_per_s"] / 1e12
            out["measured_fma2_peak"] = round(m, 3)
            out["frac_of_measured_fma2"] = round(achieved / m, 4)
        return out
    if w["rhs"] in MUFU_PER_STEP and rates:
        n_exp, n_rcp = MUFU_PER_STEP[w["rhs"]]
        work = (n_exp + n_rcp) * n_work * steps_per_launch
        achieved = work / (avg_launch_ms / 1e3) / 1e12
        # the exp and reciprocal operations share the multi-function unit: the mix's time
        # per step is the sum of the two kinds' times at their measured rates
        peak = (n_exp + n_rcp) / (n_exp / rates["ex2_per_s"] + n_rcp / rates["rcp_per_s"]) / 1e12
        return {"bound": "mufu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "Tops/s",
                "frac": round(achieved / peak, 4),
                "peak_basis": f"measured ex2 {rates['ex2_per_s']:.3e}/s and rcp {rates['rcp_per_s']:.3e}/s "
                              f"(ff_pipe_rate) for the mix {n_exp} exp + {n_rcp} reciprocals",
                "work_per_particle_step": f"{n_exp + n_rcp} MUFU operations counted from the equations"}
    return None


def measure_workload(args, w, dev, stream, steps, warmup, with_e2e, world, kahan=False, rates=None, reset=False,
                     clocks_enabled=True):
    """Time whole runs of one workload (re-seed, then its frames of RK4 steps with the
    projection and count splat of the frames that draw) and return the bench record."""
    import torch
    import paper_1505_00344_gb300 as ff

    P = total_particles(w)
    view = ff.make_view(**w["view"])
    H, Wd = w["view"]["height"], w["view"]["width"]
    sysobj = ff.System.from_workload(w, kahan=kahan, stream=stream)
    if args.ppt or args.block or args.blocks_per_sm:
        sysobj.set_launch(args.ppt, args.block, args.blocks_per_sm, 0)  # 0: the library's default
    if reset:
        rs = w["reset"]
        sysobj.set_reset(rs["lo"], rs["hi"], rs["t_max"], rs["check_every"])
    image = torch.zeros((H, Wd), dtype=torch.int32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > 129 MB L2
    every = w.get("splat_every_frame", False)
    schedule = {int(k): v for k, v in w.get("schedule", {}).items()}
    base_params = list(w["params"])
    counted = {"launches": 0, "record": None}

    def job(events=None, count=False):
        """One whole workload run."""
        sysobj.reset()
        sysobj.set_params(base_params)
        launches = len(w["groups"])  # the seed kernel, once per group
        for f in range(w["frames"]):
            if f in schedule:
                sysobj.set_params(schedule[f])
            if events is not None:
                events.append(torch.cuda.Event(enable_timing=True))
                events[-1].record()
            if every or f == w["frames"] - 1:
                # one frame: step + project + splat (the library fuses the splat into the
                # integrator's last launch where its kernel has the epilogue)
                sysobj.step_splat(w["steps_per_frame"], w["dt"], view, image)
            else:
                sysobj.step(w["steps_per_frame"], w["dt"])
            if events is not None:
                events.append(torch.cuda.Event(enable_timing=True))
                events[-1].record()
            if count:
                rec = sysobj.last_launch()  # what the library launched, not a guess
                launches += rec["integrator_launches"] + rec["splat_launches"]
                if every or f == w["frames"] - 1:
                    counted["record"] = rec
        if count:
            counted["launches"] = launches

    for k in range(max(1, warmup)):
        job(count=(k == 0))
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index, enabled=clocks_enabled)
    step_ms, int_ms = [], []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(steps):
        flush.zero_()  # evict the state and image from L2 between timed steps
        ev = []
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record()
        job(ev)
        s1.record()
        torch.cuda.synchronize()
        step_ms.append(s0.elapsed_time(s1))
        for a, b in zip(ev[0::2], ev[1::2]):
            int_ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()

    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / steps
    value = world * P * total_steps(w) / (ms_per_step / 1e3)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    max_mhz = (clk or {}).get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or 2070.0
    rec = counted["record"] or {}
    fused = bool(rec.get("fused_splat"))
    n_work = (P + 3) // 4 * 4
    avg_int_ms = statistics.mean(int_ms)
    # a frame's launch window holds one integrator launch when the call was not split
    per_launch = w["steps_per_frame"] // max(1, rec.get("integrator_launches", 1))
    roof = roofline_for(w, n_work, avg_int_ms * per_launch / w["steps_per_frame"], per_launch, sms, max_mhz, rates,
                        kahan)
    if roof:
        kernel = rec.get("kernel", "")
        # DRAM bytes come from the committed ncu record, which is of the fused kernel on the full
        # lorenz_4M frame: only that workload and kernel, on the same sources, gets it
        recorded = (w["name"] == "lorenz_4M" and fused and "lorenz_rk4_x2u_kernel<false, 2, true>" in kernel
                    and not args.particles and not args.frame_steps)
        roof.update({"traffic": traffic_from_profile(kernel_source_hash()) if recorded else None,
                     "kernel": kernel, "grid": rec.get("grid"), "block": rec.get("block"),
                     "kernel_reported_by": "ff_last_launch",
                     "algorithmic_bytes_per_launch": 2 * 4 * w["dim"] * n_work,
                     "launch_window": ("ff_step_splat: image clear + integrator with fused splat" if fused else
                                       "ff_step_splat: integrator + splat kernel" if every else
                                       "ff_step: integrator"),
                     "avg_launch_ms": round(avg_int_ms, 4)})
        if clk and roof["bound"] == "alu":
            roof["frac_at_sampled_clock"] = round(
                roof["achieved"] / (sms * FP32_LANES_PER_SM * 2 * clk["sm_mhz"] * 1e6 / 1e12), 4)
    out = {"value": value, "ms_per_step": ms_per_step, "frames_per_s": w["frames"] / (ms_per_step / 1e3),
           "gpu_launches": counted["launches"] * steps, "wall_s_timed_region": wall, "roofline": roof,
           "clocks": clk or {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": [],
                             "note": "not sampled (--no-clocks)" if not clocks_enabled else
                             "timed region shorter than the 200 ms sampling interval"},
           "particles": P, "steps": steps}
    if with_e2e:
        out["e2e"] = e2e_ours(args, sysobj, w, view, image, P, world, dev, reps=min(steps, 5))
    sysobj.close()
    return out


def run_ours(args, rank, world, local):
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream().cuda_stream
    w = workload_for(args, rank, world)
    rates = pipe_rates(local)
    m = measure_workload(args, w, dev, stream, args.steps, args.warmup, not args.no_e2e, world, kahan=args.kahan,
                         rates=rates, reset=args.reset, clocks_enabled=not args.no_clocks)
    P = m["particles"]
    Wd, H = w["view"]["width"], w["view"]["height"]
    result = {
        "metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["name"], "particles_per_gpu": P, "groups": [
            {"count": g["count"], "direction": g["direction"]} for g in w["groups"]],
            "rk4_steps_per_job": total_steps(w), "frames": w["frames"], "steps_per_frame": w["steps_per_frame"],
            "dt": w["dt"], "image": f"{Wd}x{H}", "kahan": bool(args.kahan), "reset": bool(args.reset),
            "profiling_case": bool(args.particles or args.frames),
            "l2": "flushed (256 MB write) before every timed step", "parallelism": "dp%d-weak-shards" % world,
            "launch": {"particles_per_thread": args.ppt or "library default", "block": args.block or "library default",
                       "blocks_per_sm": args.blocks_per_sm}},
        "frames_per_s": m["frames_per_s"],
        "gpu_launches": m["gpu_launches"],
        "wall_s_timed_region": m["wall_s_timed_region"],
        "clocks": m["clocks"],
        "pipe_rates": rates,
    }
    if m["roofline"]:
        result["roofline"] = m["roofline"]
    if "e2e" in m:
        result["e2e"] = m["e2e"]
    default_run = (w["name"] == "lorenz_4M" and not (args.kahan or args.reset or args.particles or args.frames
                                                     or args.frame_steps or args.ppt or args.block
                                                     or args.blocks_per_sm or args.no_extras))
    if default_run:
        # the gradient half of the metric and the other workloads, each with its own clocks; on one
        # GPU a sub-record that fails says so in its place and leaves the headline standing (with
        # several ranks an error propagates: the records take max-over-ranks collectives, which a
        # rank that gave up would leave the others waiting in)
        def sub(fn):
            if world > 1:
                return fn()
            try:
                return fn()
            except Exception as e:  # noqa: BLE001 -- reported in the record
                return {"error": f"{type(e).__name__}: {e}"}

        def batch_records():
            # every rank runs the whole batch: the job's value is this rank's times the ranks
            recs = {"forward": batch_timings("mixed_batch256", 500, 3, 1, dev, stream,
                                             clocks_enabled=not args.no_clocks),
                    "adjoint": batch_adjoint_timings("mixed_batch256", 200, 100, 2, 1, dev, stream,
                                                     clocks_enabled=not args.no_clocks)}
            for r in recs.values():
                r["value"] *= world
            return recs

        def workload_record(name, steps):
            wl = W.shard(W.workload(name), rank, world)
            r = measure_workload(args, wl, dev, stream, steps, 2 if name == "hh3_1M" else 3, not args.no_e2e, world,
                                 rates=rates, clocks_enabled=not args.no_clocks)
            r["metric"] = METRIC
            r["unit"] = UNIT
            return r

        result["adjoint"] = sub(lambda: adjoint_record(args, w, dev, stream, world))
        result["adjoint_hh3_1M"] = sub(lambda: adjoint_record(args, W.shard(W.workload("hh3_1M"), rank, world), dev,
                                                              stream, world, n=1000, K=100))
        # the batched systems: forward (one graph launch per step call) and gradients
        result["batch_mixed256"] = sub(batch_records)
        result["workloads"] = {name: sub(lambda name=name, steps=steps: workload_record(name, steps))
                               for name, steps in (("hh3_1M", 2), ("lorenz_bif_8M", 3), ("wc_4k", 10))}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w)
    if world > 1:
        torch.distributed.destroy_process_group()
    return result


def e2e_ours(args, sysobj, w, view, image, P, world, dev, reps=5):
    """Same metric through the public API with host buffers: each step uploads the initial state
    from pinned host memory (ff_set_state) and reads the final image back to pinned host memory
    (ff_project_splat with a host image)."""
    import torch

    dim = w["dim"]
    H, Wd = w["view"]["height"], w["view"]["width"]
    sysobj.reset()
    x0 = torch.empty((dim, P), dtype=torch.float32, pin_memory=True)
    sysobj.get_state(x0.numpy())
    host_img = torch.zeros((H, Wd), dtype=torch.int32, pin_memory=True)
    every = w.get("splat_every_frame", False)
    schedule = {int(k): v for k, v in w.get("schedule", {}).items()}

    def job():
        sysobj.set_state(x0)  # upload the initial state (also clears the Kahan compensation)
        sysobj.set_params(w["params"])
        for f in range(w["frames"]):
            if f in schedule:
                sysobj.set_params(schedule[f])
            sysobj.step(w["steps_per_frame"], w["dt"])
            last = f == w["frames"] - 1
            if last:
                sysobj.project_splat(view, host_img.numpy())
            elif every:
                sysobj.project_splat(view, image)

    job()
    torch.cuda.synchronize()
    times = []
    for _ in range(max(1, min(args.steps, reps))):
        t0 = time.perf_counter()
        job()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = max_over_ranks(statistics.mean(times), dev)
    return {"value": world * P * total_steps(w) / t, "unit": UNIT, "h2d_bytes_per_step": 4 * dim * P,
            "d2h_bytes_per_step": 4 * H * Wd, "steps": len(times)}


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------
def oracle_sample_run(w, particles, steps, threads=None):
    """FP64 oracle on a bounded sample: the first particles of each group (proportional),
    `steps` RK4 steps, then the x-z splat. Returns (particle-steps, seconds, threads)."""
    import oracle

    ws = W.scaled(w, particles)
    x0 = np.concatenate([oracle.seed_group(ws["dim"], g["lo"], g["hi"], g["seed"], count=g["count"])
                         for g in ws["groups"]], axis=1)
    h = np.concatenate([np.full(g["count"], g["direction"] * ws["dt"]) for g in ws["groups"]])
    n = x0.shape[1]
    rid = W.RHS_IDS[ws["rhs"]]
    v = ws["view"]
    t0 = time.perf_counter()
    x, used = oracle.integrate_parallel(rid, x0, ws["params"], h, steps, threads=threads)
    xf = x.astype(np.float32)
    if v["ndim_view"] == 2 and max(v["axes"]) < ws["dim"]:
        oracle.splat2d(xf[v["axes"][0]], xf[v["axes"][1]], v["lo"], v["hi"], v["width"], v["height"])
    dt = time.perf_counter() - t0
    return n * steps, dt, used


def cpu_baseline(w):
    threads = os.cpu_count() or 1
    # a quick probe sizes the sample to about 15 s of total CPU work
    work, t, _ = oracle_sample_run(w, 4096, 200, threads=1)
    rate1 = work / t
    steps = w["steps_per_frame"]
    particles = int(min(4_194_304, max(threads * 4096, 15.0 * rate1 / steps)))
    work, t, used = oracle_sample_run(w, particles, steps, threads=threads)
    job = total_particles(w) * w["frames"] * w["steps_per_frame"]  # particle-steps of the whole job
    return {"value": work / t, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{particles} particles of {w['name']} (groups in proportion) x {steps} RK4 steps "
                      f"+ x-z splat, FP64 oracle, {used} threads on disjoint particle ranges",
            "per_core": rate1, "per_core_sample": "4096 particles x 200 RK4 steps + splat, one thread",
            "full_job_s": job / (work / t)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w = W.workload(args.workload)
    threads = os.cpu_count() or 1
    steps = w["steps_per_frame"]
    particles = min(total_particles(w), 262_144)
    for _ in range(args.warmup):
        oracle_sample_run(w, particles // 8, steps, threads=threads)
    times = []
    work = 0
    for _ in range(args.steps):
        work, t, used = oracle_sample_run(w, particles, steps, threads=threads)
        times.append(t)
    value = work / statistics.mean(times)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w["name"], "sample_particles": particles,
                                            "rk4_steps_per_step": steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": f"{particles} particles x {steps} RK4 steps + splat per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def adjoint_timings(w, n, K, steps, warmup, dev, stream, clocks_enabled=True):
    """Plain forward, taped forward and adjoint sweep of n RK4 steps (checkpoint every K) for
    the workload's particles: gradients of L = (1/P) sum |x(T) - t|^2 w.r.t. the initial
    states and parameters.  CUDA events on the system's stream; median of `steps` runs."""
    import torch
    import paper_1505_00344_gb300 as ff

    P, dim, dt = total_particles(w), w["dim"], w["dt"]
    s = ff.System.from_workload(w, stream=stream)
    x0 = torch.empty((dim, P), dtype=torch.float32, device=dev)
    s.get_state(x0)
    target = torch.empty_like(x0).uniform_(-20.0, 20.0)
    dx0 = torch.empty_like(x0)
    n_params = len(w["params"])
    grad = torch.empty_like(x0)

    def timed(fn):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    def plain():
        s.set_state(x0)
        s.step(n, dt)

    def taped():
        s.set_state(x0)
        s.tape_begin(K, n)
        s.step(n, dt)

    def backward():
        s.backward(grad, dx0, n_params)

    def sweep():  # taped forward, loss gradient, reverse sweep
        tf = timed(taped)
        xT = torch.empty_like(x0)
        s.get_state(xT)
        torch.mul(xT - target, 2.0 / P, out=grad)
        return tf, timed(backward)

    # warm-up runs every kernel of the timed steps once (the first launch of a kernel also loads it)
    for _ in range(max(1, warmup)):
        plain()
        sweep()
    clocks = ClockSampler(dev.index, enabled=clocks_enabled)
    t_plain = [timed(plain) for _ in range(max(1, steps))]
    t_fwd, t_bwd = [], []
    for _ in range(max(1, steps)):
        tf, tb = sweep()
        t_fwd.append(tf)
        t_bwd.append(tb)
    clk = clocks.stop()
    s.tape_end()
    s.close()
    units = P * n
    med = statistics.median
    return {"value": units / (med(t_bwd) / 1e3), "unit": UNIT, "particles": P, "rk4_steps": n,
            "checkpoint_every": K, "plain_forward": units / (med(t_plain) / 1e3),
            "taped_forward": units / (med(t_fwd) / 1e3), "backward_over_plain_time": med(t_bwd) / med(t_plain),
            "ms": {"plain": med(t_plain), "taped_forward": med(t_fwd), "backward": med(t_bwd)},
            "clocks": clk or {"sm_mhz": None, "samples": 0, "reasons": [],
                              "note": "timed region shorter than the 200 ms sampling interval"}}


def adjoint_record(args, w, dev, stream, world, n=2000, K=100):
    """The gradient half of the metric inside the default bench line: the workload's particles,
    n RK4 steps, checkpoint every K (lorenz_4M: 2,000 and 100)."""
    r = adjoint_timings(w, n, K, 3, 2, dev, stream, clocks_enabled=not args.no_clocks)
    r["metric"] = "adjoint particle-RK4-steps/sec (gradients w.r.t. initial states and parameters)"
    r["loss"] = "mean squared distance of final states to random targets"
    r["dtype"] = "f32 (FP64 parameter sums)"
    r["value"] *= world
    return r


def run_adjoint(args, rank, world, local):
    """Gradients of L = (1/P) sum |x(T) - t|^2 w.r.t. initial states and parameters for the
    workload's particles over --adjoint-steps RK4 steps (checkpoint every --checkpoint-every):
    particle-steps/s of the plain forward, the taped forward and the adjoint sweep."""
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload_for(args, rank, world)
    r = adjoint_timings(w, args.adjoint_steps, args.checkpoint_every, args.steps, args.warmup, dev,
                        torch.cuda.current_stream().cuda_stream, clocks_enabled=not args.no_clocks)
    return {"metric": "adjoint particle-RK4-steps/sec (gradients w.r.t. initial states and parameters)",
            "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms"]["backward"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (FP64 parameter sums)", "data": "synthetic",
            "config": {"workload": w["name"], "particles": r["particles"], "rk4_steps": r["rk4_steps"],
                       "checkpoint_every": r["checkpoint_every"],
                       "loss": "mean squared distance of final states to random targets"},
            "plain_forward": r["plain_forward"], "taped_forward": r["taped_forward"],
            "backward_over_plain_time": r["backward_over_plain_time"], "ms": r["ms"], "clocks": r["clocks"]}


def _timed_on_stream(fn):
    import torch
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    e.record()
    torch.cuda.synchronize()
    return a.elapsed_time(e)


def batch_timings(name, n, steps, warmup, dev, stream, clocks_enabled=True):
    """ff_batch_step of n RK4 steps over a batched workload (one graph launch, autotuned
    launch shapes) against stepping the same systems one after the other with ff_step."""
    import paper_1505_00344_gb300 as ff

    ws = W.batch_workload(name)
    systems = [ff.System.from_workload(w, stream=stream) for w in ws]
    dts = [w["dt"] for w in ws]
    units = sum(total_particles(w) for w in ws) * n
    b = ff.Batch(systems, stream=stream)
    b.autotune(dts, trial_steps=max(8, min(64, n // 10)))

    def batched():
        b.step(n, dts)

    def one_by_one():
        for s_, dt in zip(systems, dts):
            s_.step(n, dt)

    for _ in range(warmup):
        batched()
    clocks = ClockSampler(dev.index, enabled=clocks_enabled)
    tb = [_timed_on_stream(batched) for _ in range(max(1, steps))]
    clk = clocks.stop()
    to = [_timed_on_stream(one_by_one) for _ in range(max(1, steps))]
    launch = b.describe().strip().split("\n")
    b.close()
    for s_ in systems:
        s_.close()
    med = statistics.median
    return {"metric": "particle-RK4-steps/sec (batched systems)", "value": units / (med(tb) / 1e3), "unit": UNIT,
            "workload": name, "systems": len(ws), "particles": units // n, "rk4_steps": n, "ms": med(tb),
            "launch": launch, "one_by_one": units / (med(to) / 1e3), "speedup_vs_one_by_one": med(to) / med(tb),
            "gpu_launches": len({(w["rhs"], w["method"]) for w in ws}),  # one kernel per family in the graph
            "clocks": clk or {"sm_mhz": None, "samples": 0, "reasons": [],
                              "note": "timed region shorter than the 200 ms sampling interval"}}


def batch_adjoint_timings(name, n, K, steps, warmup, dev, stream, clocks_enabled=True):
    """The differentiable batched ensemble: a taped ff_batch_step of n RK4 steps (checkpoint
    every K) and one ff_batch_backward, gradients of L = sum_s (1/P_s) sum_i |x_i(T) - t_i|^2
    w.r.t. every member's initial states and parameters; against the plain batched forward."""
    import torch
    import paper_1505_00344_gb300 as ff

    ws = W.batch_workload(name)
    systems = [ff.System.from_workload(w, stream=stream) for w in ws]
    dts = [w["dt"] for w in ws]
    b = ff.Batch(systems, stream=stream)
    b.autotune(dts, trial_steps=16)
    x0, tgt = [], []
    for k, (s, w) in enumerate(zip(systems, ws)):
        P, dim = total_particles(w), w["dim"]
        x = torch.empty((dim, P), dtype=torch.float32, device=dev)
        s.get_state(x)
        x0.append(x)
        g = torch.Generator(device=dev).manual_seed(7000 + k)
        lo = torch.tensor(w["groups"][0]["lo"], dtype=torch.float32, device=dev)[:, None]
        hi = torch.tensor(w["groups"][0]["hi"], dtype=torch.float32, device=dev)[:, None]
        tgt.append(lo + (hi - lo) * torch.rand((dim, P), generator=g, device=dev))
    units = sum(total_particles(w) for w in ws) * n

    def restore():
        for s, x in zip(systems, x0):
            s.set_state(x)

    grads = [torch.empty_like(x) for x in x0]
    outs = [torch.empty_like(x) for x in x0]

    def loss_grads():
        for s, x, t, g in zip(systems, x0, tgt, grads):
            s.get_state(g)
            g.sub_(t).mul_(2.0 / x.shape[1])

    t_plain, t_fwd, t_bwd = [], [], []
    clocks = None
    for it in range(warmup + max(1, steps)):
        if it == warmup:
            clocks = ClockSampler(dev.index, enabled=clocks_enabled)
        restore()
        tp = _timed_on_stream(lambda: b.step(n, dts))
        restore()
        b.tape_begin(K, n)
        tf = _timed_on_stream(lambda: b.step(n, dts))
        loss_grads()
        tb = _timed_on_stream(lambda: b.backward(grads, outs))
        b.tape_end()
        if it >= warmup:
            t_plain.append(tp)
            t_fwd.append(tf)
            t_bwd.append(tb)
    clk = clocks.stop()
    launch = b.describe().strip().split("\n")
    b.close()
    for s_ in systems:
        s_.close()
    med = statistics.median
    return {"metric": "adjoint particle-RK4-steps/sec (batched ensemble, gradients w.r.t. all initial states "
                      "and parameters)",
            "value": units / (med(t_bwd) / 1e3), "unit": UNIT, "workload": name, "systems": len(ws),
            "particles": units // n, "rk4_steps": n, "checkpoint_every": K,
            "loss": "sum over systems of the mean squared endpoint distance to seeded targets",
            "launch": launch, "plain_forward": units / (med(t_plain) / 1e3),
            "taped_forward": units / (med(t_fwd) / 1e3), "backward_over_plain_time": med(t_bwd) / med(t_plain),
            "ms": {"plain": med(t_plain), "taped_forward": med(t_fwd), "backward": med(t_bwd)},
            "clocks": clk or {"sm_mhz": None, "samples": 0, "reasons": [],
                              "note": "timed region shorter than the 200 ms sampling interval"}}


def run_batch_adjoint(args, rank, world, local):
    """Command-line form of batch_adjoint_timings (--batch NAME --adjoint)."""
    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    r = batch_adjoint_timings(args.batch, args.adjoint_steps, args.checkpoint_every, args.steps, args.warmup, dev,
                              torch.cuda.current_stream().cuda_stream, clocks_enabled=not args.no_clocks)
    return {"metric": r["metric"], "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"]["backward"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 parameter sums)", "data": "synthetic",
            "config": {"workload": args.batch, "systems": r["systems"], "particles": r["particles"],
                       "rk4_steps": r["rk4_steps"], "checkpoint_every": r["checkpoint_every"], "loss": r["loss"],
                       "launch": r["launch"]},
            "plain_forward": r["plain_forward"], "taped_forward": r["taped_forward"],
            "backward_over_plain_time": r["backward_over_plain_time"], "ms": r["ms"], "clocks": r["clocks"]}


def run_batch(args, rank, world, local):
    """Command-line form of batch_timings (--batch NAME)."""
    import torch

    torch.cuda.set_device(local)
    r = batch_timings(args.batch, args.batch_steps, args.steps, args.warmup, torch.device("cuda", local),
                      torch.cuda.current_stream().cuda_stream, clocks_enabled=not args.no_clocks)
    return {"metric": r["metric"], "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.batch, "systems": r["systems"], "particles": r["particles"],
                       "rk4_steps": r["rk4_steps"], "launch": r["launch"]},
            "one_by_one": r["one_by_one"], "speedup_vs_one_by_one": r["speedup_vs_one_by_one"],
            "gpu_launches": r["gpu_launches"], "clocks": r["clocks"]}


def run_sprites(args, rank, world, local):
    """The workload's frame loop with soft sprites (radius --sprites) instead of the count
    splat: frames/s of ff_step + ff_project_sprites, and the sprite kernel's own rate."""
    import math

    import torch
    import paper_1505_00344_gb300 as ff

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload_for(args, rank, world)
    stream = torch.cuda.current_stream().cuda_stream
    s = ff.System.from_workload(w, stream=stream)
    v = w["view"]
    Wd, Hd = v["width"], v["height"]
    view = ff.make_view(**v)
    groups = len(w["groups"])
    palette = [[1.0, 0.55, 0.15, 1.0], [0.2, 0.45, 1.0, 1.0], [0.3, 1.0, 0.4, 1.0], [1.0, 0.3, 0.8, 1.0]]
    technique = {"auto": ff.FF_SPRITE_AUTO, "direct": ff.FF_SPRITE_DIRECT, "tiled": ff.FF_SPRITE_TILED}[
        args.sprite_technique]
    sprite = ff.make_sprite(args.sprites, 0.05, [palette[g % 4] for g in range(groups)], technique)
    img = torch.zeros((Hd, Wd, 4), dtype=torch.float32, device=dev)
    counts = torch.zeros((Hd, Wd), dtype=torch.int32, device=dev)
    frames = args.frames or w["frames"]
    n, dt = w["steps_per_frame"], w["dt"]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    events = []

    def job(record):
        s.reset()
        for _ in range(frames):
            s.step(n, dt)
            if record:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                s.project_sprites(view, sprite, img)
                b.record()
                events.append((a, b))
            else:
                s.project_sprites(view, sprite, img)

    for _ in range(args.warmup):
        job(False)
    ts = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        job(True)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    sprite_ms = statistics.median([x.elapsed_time(y) for x, y in events])
    # fragments of the last frame: drawn particles (the count splat) x the lattice points of a disc
    s.project_splat(view, counts)
    drawn = int(counts.sum().item())
    frags = drawn * math.pi * args.sprites ** 2
    med = statistics.median(ts)
    P = total_particles(w)
    return {"metric": "frames/sec (RK4 frames with soft-sprite rendering)", "value": frames / (med / 1e3),
            "unit": "frames/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": med,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "particles": P, "frames": frames, "steps_per_frame": n,
                       "sprite_radius": args.sprites, "sprite_technique": args.sprite_technique,
                       "image": [Hd, Wd, 4], "l2": "256 MB flush between steps"},
            "particle_steps_per_s": P * n * frames / (med / 1e3),
            "sprite_kernel": {"ms_per_frame": sprite_ms, "drawn_particles": drawn,
                              "fragments_per_frame_est": frags,
                              "fragments_per_s": frags / (sprite_ms / 1e3),
                              "reduction_GBps": 16.0 * frags / (sprite_ms / 1e3) / 1e9,
                              "share_of_frame": sprite_ms * frames / med},
            "gpu_launches": (2 if args.sprite_technique == "direct" else 5) * frames}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.batch and args.adjoint:
        out = run_batch_adjoint(args, rank, world, local)
    elif args.adjoint:
        out = run_adjoint(args, rank, world, local)
    elif args.batch:
        out = run_batch(args, rank, world, local)
    elif args.sprites > 0:
        out = run_sprites(args, rank, world, local)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
