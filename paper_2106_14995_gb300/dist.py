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


def shard_by_cost(costs, rank: int, world: int) -> tuple:
    """Contiguous range [start, end) of the problems for ``rank`` with about equal
    predicted cost per rank: rank r ends at the first problem where the running cost
    reaches (r + 1) / world of the total, so each rank's cost is at most total / world
    plus one problem's.  ``costs[p]`` >= 0 predicts problem p's solve time: n^3 for
    dense problems of mixed size n (the factorizations dominate), or, for problems
    solved again warm started (the ADMM's branches), the iteration count of the previous
    solve.  Equal-count splits in index order, as in Sec. 6.2, leave ranks unevenly
    loaded when the problems differ in size or difficulty: Table 5 reports 9-47 % mean
    imbalance for the ADMM's branch batches split that way."""
    import numpy as np
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    c = np.asarray(costs, dtype=np.float64).ravel()
    if c.size and (not np.all(np.isfinite(c)) or c.min() < 0):
        raise ValueError("costs must be finite and >= 0")
    cum = np.cumsum(c)
    total = float(cum[-1]) if c.size else 0.0
    if total == 0.0:
        return shard(c.size, rank, world)

    def cut(r):
        # problems [0, cut(r)) belong to ranks < r
        if r <= 0:
            return 0
        if r >= world:
            return int(c.size)
        return int(np.searchsorted(cum, total * r / world, side="left")) + 1

    start, end = cut(rank), cut(rank + 1)
    return min(start, c.size), min(max(end, start), c.size)


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
