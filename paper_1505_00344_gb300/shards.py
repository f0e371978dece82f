"""One ensemble split across GPUs, and the one exchange per frame that joins it.

The particles of an ensemble are independent (the paper integrates each on its own
work-item, Appendix A), so the ensemble is split by particle index into contiguous
ranges, one per rank (one process per GPU).  Each rank seeds exactly its range --
``ff_seed_particles_slice`` draws the random numbers the whole system would draw for
those particles, and ``ff_set_particle_param_slice`` gives them the whole ensemble's
linspace values -- integrates it and splats it into an image of its own.

The only data exchange is a sum over ranks: the uint32 count images of a frame (an
exact integer sum, so the reduced image is the unsplit ensemble's image bit for bit)
and, for gradients, the FP64 parameter gradients dL/dp (the unsplit sum up to the
order of its FP64 additions).  dL/dx0 of a particle is computed by the rank holding
it.  The sums go through ``torch.distributed`` (NCCL between GPUs, gloo on CPU).

This module holds index bookkeeping and the reduction calls only; every step of the
path runs in the CUDA library.
"""
from __future__ import annotations

from . import System


def split_range(total: int, rank: int, world: int, align: int = 4) -> tuple[int, int]:
    """Particle indices [a, b) of `rank`: contiguous ranges in rank order that cover
    [0, total), with inner boundaries on multiples of `align` (so each rank's groups
    keep the alignment the packed integrators want)."""
    if world < 1 or not 0 <= rank < world or align < 1 or total < 0:
        raise ValueError("bad split arguments")
    units = -(-total // align)
    a = min(total, (units * rank // world) * align)
    b = min(total, (units * (rank + 1) // world) * align)
    return a, b


def group_slices(counts, a: int, b: int):
    """For groups of the given sizes laid out consecutively, the part of each inside
    [a, b): a list of (group index, first index within the group, count, group size),
    skipping groups that do not meet the range."""
    out = []
    start = 0
    for gi, n in enumerate(counts):
        lo, hi = max(a, start), min(b, start + n)
        if hi > lo:
            out.append((gi, lo - start, hi - lo, n))
        start += n
    return out


def shard_system(w: dict, rank: int, world: int, stream=None, kahan: bool = False, align: int = 4):
    """The system of `rank` for workload `w` split across `world` ranks.

    Returns (system, groups, (a, b)): the System (None if the rank's range is empty),
    the global index of each of its local groups, and its particle range."""
    counts = [g["count"] for g in w["groups"]]
    total = sum(counts)
    a, b = split_range(total, rank, world, align)
    if b <= a:
        return None, [], (a, b)
    s = System(w["rhs"], w["params"], b - a, dim=w["dim"], method=w.get("method", "rk4"), kahan=kahan,
               stream=stream)
    groups = []
    for gi, first, count, size in group_slices(counts, a, b):
        g = w["groups"][gi]
        s.seed_slice(count, first, size, g["lo"], g["hi"], g["direction"], g["seed"])
        groups.append(gi)
    if "pparam" in w:
        pp = w["pparam"]
        s.set_particle_param_slice(pp["index"], pp["lo"], pp["hi"], a, total)
    return s, groups, (a, b)


def local_group_mask(mask: int, groups) -> int:
    """A view's group mask over the whole ensemble's groups, as the mask over a shard's
    local groups (local group i is global group groups[i])."""
    out = 0
    for i, gi in enumerate(groups):
        if (mask >> gi) & 1:
            out |= 1 << i
    return out


def allreduce_sum(tensor, group=None):
    """Sum `tensor` over all ranks in place (one collective) and return it: uint32
    count images (as int32 tensors; two's-complement addition is the same bits) or
    FP64 gradient vectors."""
    import torch.distributed as dist

    dist.all_reduce(tensor, op=dist.ReduceOp.SUM, group=group)
    return tensor
