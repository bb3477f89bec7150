"""Multi-rank helpers for the batched solve (one process per GPU).

The TRON batch partitions into independent problems, so ranks exchange nothing on the
data path: each rank solves its own problems, and only the timing is combined (the
maximum over ranks, one scalar all-reduce) when throughput is reported.
"""
from __future__ import annotations


def shard(total: int, rank: int, world: int) -> tuple:
    """Contiguous, balanced range [start, end) of ``total`` problems for ``rank``."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(int(total), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over all ranks (identity without an initialised group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_throughput(units_per_rank: int, world: int, steps: int,
                            max_elapsed_ms: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest rank's time."""
    return world * units_per_rank * steps / (max_elapsed_ms * 1e-3)
