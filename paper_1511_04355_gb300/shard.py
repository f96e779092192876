"""Frequency sharding over ranks (one process per GPU).

The frequency solves are independent (Sec. 2.2: one boundary-element solve per sampling
frequency), so N GPUs split a frequency grid into N contiguous shards and solve them with no
exchange on the data path; only the timing is reduced (maximum over ranks).  Host-side
arithmetic only: no GPU code lives here.
"""
from __future__ import annotations


def shard_bounds(n_total: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous shard of n_total items; shard sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard(seq, rank: int, world: int):
    """rank's contiguous part of a sequence (numpy array, list, tensor)."""
    lo, hi = shard_bounds(len(seq), rank, world)
    return seq[lo:hi]


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a per-rank number over all ranks of the default process group (the value
    itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    if seconds_max <= 0:
        raise ValueError("non-positive time")
    return units_per_rank * world / seconds_max
