"""Packet-id sharding across ranks (one process per GPU).

Packets are independent and each one's random stream is keyed by its id
(Philox counter), so a multi-GPU run is a partition of the id space with no
exchange inside the walk. The only exchange is the final sum of the
tallies, done once after the last step.
"""
from __future__ import annotations


def step_range(step: int, rank: int, world: int, per_rank: int, first: int = 0):
    """Ids [lo, lo + per_rank) that `rank` runs at `step`: step-major, so the
    ranks of one step together cover one contiguous chunk of the job."""
    if not (0 <= rank < world) or per_rank < 0 or step < 0:
        raise ValueError("bad shard arguments")
    lo = first + (step * world + rank) * per_rank
    return lo, per_rank


def max_over_ranks(value: float) -> float:
    """Largest value across ranks (timings); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(tensor):
    """In-place sum of a tally tensor across ranks (the one exchange step)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(tensor, op=dist.ReduceOp.SUM)
    return tensor


def reduce_tallies(tensors):
    """The job's one exchange: sum each rank's tallies (escaped spectrum,
    scattering map, ...) in place, so that every rank holds the tallies of
    the whole job. Integer tallies sum exactly; FP64 ones up to rounding."""
    for t in tensors:
        if t is not None:
            sum_over_ranks(t)
    return tensors
