"""Host-side logic of running independent problems on several GPUs (replicas).

Independent images (or alpha values) share nothing, so several GPUs run them
with no data-path exchange: each rank takes its own items, times its own
work, and only the timing and the item counts are combined (a maximum and a
sum over the ranks). Works with any torch.distributed backend (NCCL on GPUs,
gloo on the CPU); without an initialised process group it is the one-rank case.
"""
from __future__ import annotations


def shard(sizes, rank: int, world: int) -> list[int]:
    """Indices of the items this rank takes: largest first, each to the rank
    with the least work so far (ties to the lower rank); deterministic, so
    every rank computes the same split without communicating."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank must be in [0, world)")
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += sizes[i]
        if r == rank:
            mine.append(i)
    return sorted(mine)


def _dist():
    try:
        import torch.distributed as dist
    except ImportError:  # pragma: no cover
        return None
    return dist if dist.is_available() and dist.is_initialized() else None


def reduce_over_ranks(value: float, op: str, device=None) -> float:
    """max or sum of a float over all ranks (the value itself with one rank)."""
    dist = _dist()
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units_local: float, ms_local: float, device=None) -> float:
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    units = reduce_over_ranks(units_local, "sum", device)
    ms = reduce_over_ranks(ms_local, "max", device)
    return 1000.0 * units / ms
