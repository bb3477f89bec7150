"""The multi-rank path on CPU: two gloo ranks shard a batch of independent problems,
solve their shards (with the oracle: no GPU here), and combine only the timing.  The
union of the shards must be the whole batch, each problem solved once, with the
results of the single-process solve; the reported time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2106_14995_gb300 import dist as xdist


def test_shard_covers_everything_once():
    for total in (0, 1, 7, 100, 1001):
        for world in (1, 2, 3, 8):
            ranges = [xdist.shard(total, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == total
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0 and a1 >= a0
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        xdist.shard(10, 2, 2)


def test_shard_by_cost_balances_mixed_sizes():
    rng = np.random.default_rng(7)
    n = rng.choice([4, 6, 8, 16, 32, 64, 128], size=5000,
                   p=[0.4, 0.2, 0.15, 0.1, 0.08, 0.05, 0.02])
    cost = n.astype(np.float64) ** 3
    for world in (1, 2, 3, 8):
        ranges = [xdist.shard_by_cost(cost, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == len(cost)
        for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
            assert a1 == b0 and a1 >= a0
        per = np.array([cost[a:b].sum() for a, b in ranges])
        assert per.max() <= cost.sum() / world + cost.max()
        # a count split of the same batch is far less even
        cnt = np.array([cost[slice(*xdist.shard(len(cost), r, world))].sum()
                        for r in range(world)])
        assert per.max() - per.min() <= cnt.max() - cnt.min() + cost.max()
    # more ranks than problems, and one dominant problem: still contiguous and covering,
    # each rank within one problem's cost of the mean
    for costs, world in (([1, 1, 1], 8), ([5, 0, 0, 0], 3), ([0, 0, 7], 4),
                         ([1e9, 1, 1, 1], 2)):
        c = np.asarray(costs, dtype=float)
        ranges = [xdist.shard_by_cost(c, r, world) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == len(c)
        assert all(a1 == b0 for (_, a1), (b0, _) in zip(ranges, ranges[1:]))
        assert max(c[a:b].sum() for a, b in ranges) <= c.sum() / world + c.max()
    # zero or empty costs fall back to the count split
    assert xdist.shard_by_cost(np.zeros(10), 1, 2) == xdist.shard(10, 1, 2)
    assert xdist.shard_by_cost([], 0, 3) == (0, 0)
    with pytest.raises(ValueError):
        xdist.shard_by_cost([1.0, -1.0], 0, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    from paper_2106_14995_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    d = synth.dense_batch(37, 8, seed_index=1)
    a, b = xdist.shard(37, rank, world)
    r = oracle.tron_batch(2, d["params"][a:b], d["l"][a:b], d["u"][a:b], d["x0"][a:b],
                          d["delta0"][a:b])
    local_ms = 10.0 * (rank + 1)  # a stand-in timing: rank 1 is the slowest
    slowest = xdist.max_over_ranks(local_ms)
    np.save(os.path.join(out_dir, f"x{rank}.npy"), r["x"])
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([slowest, a, b]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_slowest_time(tmp_path):
    import oracle
    from paper_2106_14995_gb300 import synth
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, str(tmp_path)))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    d = synth.dense_batch(37, 8, seed_index=1)
    ref = oracle.tron_batch(2, d["params"], d["l"], d["u"], d["x0"], d["delta0"])
    xs = []
    for r in range(world):
        slowest, a, b = np.load(tmp_path / f"t{r}.npy")
        assert slowest == 20.0
        xs.append(np.load(tmp_path / f"x{r}.npy"))
    np.testing.assert_array_equal(np.concatenate(xs), ref["x"])
    assert xdist.weak_scaling_throughput(37, 2, 3, 20.0) == 2 * 37 * 3 / 0.02
