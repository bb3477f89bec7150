"""Multi-rank helpers (one process per GPU).

The TRON batch partitions into independent problems, so ranks exchange nothing on the
data path: each rank solves its own problems, and only the timing is combined (the
maximum over ranks, one scalar all-reduce) when throughput is reported.  The component
ADMM partitions by buses and has one real exchange per half-iteration: the boundary
data of the cut branches (the second half of this module).
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


# ---------------------------------------------------- partitioned component ADMM
# The ADMM of Sec. 6.1 splits across GPUs by buses (Sec. 6.3 splits the branch batches
# instead, with a root rank gathering and scattering every iteration).  Each rank owns a
# block of buses, the generators on them and every branch whose from-bus it owns; per
# iteration it exchanges only the boundary data of the cut branches (from-bus and to-bus
# on different ranks):
#   1. component phase (generators, branch TRON solves) on the owned components;
#   2. branch owner -> to-bus owner: the branch-side values at the to end (p_ji, q_ji,
#      v_j^2, theta_j), 4 doubles per cut branch;
#   3. bus phase on the owned buses: the bus QP, then the multipliers and residual terms
#      of every pair whose bus-side copy the bus holds;
#   4. to-bus owner -> branch owner: the bus-side copies of those four pairs
#      (p~_ji, q~_ji, w~_j, theta~_j) and their multipliers, 8 doubles per cut branch;
#   5. one all-reduce of the two squared residual sums.
# Every quantity is computed by exactly one rank from the same inputs as in the undivided
# iteration, so the iterates are the same; only the residual sums add in another order.

def dfs_order(nbus: int, br_from, br_to, start: int = 0):
    """Buses in depth-first preorder over the branches from ``start`` (neighbours taken
    in increasing id); buses of other connected parts follow, each part from its smallest
    bus.  A contiguous block of a preorder is a union of a few subtrees of the traversal
    tree, so blocks cut few of its branches."""
    import numpy as np
    f = np.asarray(br_from, dtype=np.int64)
    t = np.asarray(br_to, dtype=np.int64)
    adj = [[] for _ in range(int(nbus))]
    for a, b in zip(f.tolist(), t.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    for lst in adj:
        lst.sort(reverse=True)  # popped from the end: smallest id first
    seen = np.zeros(int(nbus), dtype=bool)
    order = []
    for root in [int(start)] + list(range(int(nbus))):
        if seen[root]:
            continue
        stack = [root]
        while stack:
            u = stack.pop()
            if seen[u]:
                continue
            seen[u] = True
            order.append(u)
            stack.extend(v for v in adj[u] if not seen[v])
    return np.asarray(order, dtype=np.int64)


def bus_costs(net: dict, branch_cost=None):
    """Predicted work per bus: 1 for its bus update, 1 per generator on it, and the cost
    of every branch it owns (the from-bus owns a branch); ``branch_cost[k]`` is the
    previous iteration's TRON iteration count of branch k when known (the paper's Table 5
    imbalance comes from those counts differing), else 2."""
    import numpy as np
    nb = int(net["nbus"])
    f = np.asarray(net["br_from"], dtype=np.int64)
    c = np.ones(nb)
    np.add.at(c, np.asarray(net["gen_bus"], dtype=np.int64), 1.0)
    bc = (np.full(f.size, 2.0) if branch_cost is None
          else np.asarray(branch_cost, dtype=np.float64))
    if bc.shape != f.shape or (bc.size and (not np.all(np.isfinite(bc)) or bc.min() < 0)):
        raise ValueError("branch_cost must be finite, >= 0, one per branch")
    np.add.at(c, f, bc)
    return c


def partition_buses(net: dict, nparts: int, branch_cost=None):
    """part[bus] in [0, nparts): contiguous blocks of the depth-first bus order with
    about equal predicted work (``bus_costs``; each part within one bus's cost of the
    mean), so each part is a few subtrees of the traversal and few branches are cut."""
    import numpy as np
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    nb = int(net["nbus"])
    order = dfs_order(nb, net["br_from"], net["br_to"])
    cost = bus_costs(net, branch_cost)[order]
    part = np.empty(nb, dtype=np.int64)
    for r in range(nparts):
        a, b = shard_by_cost(cost, r, nparts)
        part[order[a:b]] = r
    return part


class AdmmHaloPlan:
    """Ownership and per-iteration exchange lists of one rank of a partitioned ADMM.

    ``send_values[q]`` / ``recv_copies[q]``: cut branches this rank owns whose to-bus rank
    q owns (values go out after the component phase, copies and multipliers come back
    after the bus phase); ``recv_values[q]`` / ``send_copies[q]``: cut branches rank q
    owns whose to-bus this rank owns.  Lists are in increasing branch id, so both sides
    pack and unpack in the same order."""

    VALUES = 4   # p_ji, q_ji, v_j^2, theta_j
    COPIES = 8   # their bus-side copies and multipliers

    def __init__(self, net: dict, part, rank: int):
        import numpy as np
        part = np.asarray(part, dtype=np.int64)
        self.rank = int(rank)
        self.world = int(part.max()) + 1 if part.size else 1
        f = np.asarray(net["br_from"], dtype=np.int64)
        t = np.asarray(net["br_to"], dtype=np.int64)
        g = np.asarray(net["gen_bus"], dtype=np.int64)
        self.own_bus = part == rank
        self.own_gen = part[g] == rank
        self.own_branch = part[f] == rank
        cut = part[f] != part[t]
        self.send_values, self.recv_values = {}, {}
        for q in range(self.world):
            if q == rank:
                continue
            out = np.nonzero(cut & (part[f] == rank) & (part[t] == q))[0]
            inn = np.nonzero(cut & (part[f] == q) & (part[t] == rank))[0]
            if out.size:
                self.send_values[q] = out
            if inn.size:
                self.recv_values[q] = inn
        self.recv_copies = self.send_values
        self.send_copies = self.recv_values
        self.cut_branches = int(cut.sum())

    def doubles_per_iteration(self) -> int:
        """Doubles this rank sends per iteration (both exchanges)."""
        return (self.VALUES * sum(v.size for v in self.send_values.values()) +
                self.COPIES * sum(v.size for v in self.send_copies.values()))


def _exchange(sends: dict, recvs: dict, pack, unpack, width: int, group=None):
    """Point-to-point exchange of per-branch rows with the ranks in ``sends``/``recvs``
    (torch.distributed isend/irecv; gloo on CPU, NCCL on GPUs)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    ops, bufs = [], {}
    for q, ids in sorted(recvs.items()):
        bufs[q] = torch.empty(ids.size * width, dtype=torch.float64)
        ops.append(dist.irecv(bufs[q], src=q, group=group))
    for q, ids in sorted(sends.items()):
        payload = torch.from_numpy(np.ascontiguousarray(pack(ids), dtype=np.float64).ravel())
        ops.append(dist.isend(payload, dst=q, group=group))
    for op in ops:
        op.wait()
    for q, ids in sorted(recvs.items()):
        unpack(ids, bufs[q].numpy().reshape(ids.size, width))


def partitioned_admm_step(engine, plan: AdmmHaloPlan, group=None):
    """One iteration of the partitioned component ADMM on this rank (see above).

    ``engine`` performs the rank's arithmetic on its copy of the state:
    ``phase_components(gen_mask, branch_mask)``, ``phase_buses(bus_mask) -> (pr2, du2)``,
    ``to_end_values(ids)`` / ``set_to_end_values(ids, rows)`` ([len, 4]),
    ``to_end_copies(ids)`` / ``set_to_end_copies(ids, rows)`` ([len, 8]), and ``rho``.
    Returns the primal and dual residuals of the whole network."""
    import math
    import torch
    import torch.distributed as dist
    engine.phase_components(plan.own_gen, plan.own_branch)
    _exchange(plan.send_values, plan.recv_values, engine.to_end_values,
              engine.set_to_end_values, plan.VALUES, group)
    pr2, du2 = engine.phase_buses(plan.own_bus)
    _exchange(plan.send_copies, plan.recv_copies, engine.to_end_copies,
              engine.set_to_end_copies, plan.COPIES, group)
    t = torch.tensor([pr2, du2], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and plan.world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return math.sqrt(float(t[0])), engine.rho * math.sqrt(float(t[1]))
