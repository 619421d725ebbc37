"""Host-side helpers for running one GPU per process as independent replicas.

The extraction path never exchanges data between GPUs: a batch or a request
stream shards by whole extractions.  These helpers split the work and combine
the timings (the slowest rank bounds the job) over a torch.distributed
process group; they run the same over NCCL (GPU ranks) and gloo (CPU tests).
"""

from __future__ import annotations


def shard(count: int, world: int, rank: int) -> range:
    """Contiguous share of `count` units for `rank`; shares differ by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over the default process group (itself when
    torch.distributed is not initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units_this_rank: float, ms_this_rank: float, device=None) -> tuple[float, float]:
    """(units of all ranks per second over the slowest rank's time, that time in ms)."""
    units = sum_over_ranks(units_this_rank, device)
    ms = max_over_ranks(ms_this_rank, device)
    return units / (ms * 1e-3), ms
