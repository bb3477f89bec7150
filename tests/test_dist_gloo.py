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


# ------------------------------------------------- partitioned component ADMM (Sec. 6.3)

class _OracleEngine:
    """A rank's arithmetic for the partitioned ADMM: the oracle's phases on the rank's
    full-size copy of the state (only its own and halo entries are kept current)."""

    def __init__(self, net):
        import oracle
        self.a = oracle.Admm(net)
        self.rho = 400.0
        self.to = np.asarray(net["br_to"], dtype=np.int64)

    def phase_components(self, gen_mask, br_mask):
        self.a.phase_components(gen_mask, br_mask)

    def phase_buses(self, bus_mask):
        return self.a.phase_buses(bus_mask)

    def to_end_values(self, ids):
        return self.a.arrays["br_val"][ids][:, [2, 3, 5, 7]]

    def set_to_end_values(self, ids, rows):
        self.a.arrays["br_val"][np.ix_(ids, [2, 3, 5, 7])] = rows

    def to_end_copies(self, ids):
        s = self.a.arrays
        j = self.to[ids]
        return np.concatenate([s["br_tilde"][ids][:, [2, 3]], s["bus_w"][j][:, None],
                               s["bus_th"][j][:, None], s["br_lam"][ids][:, [2, 3, 5, 7]]],
                              axis=1)

    def set_to_end_copies(self, ids, rows):
        s = self.a.arrays
        j = self.to[ids]
        s["br_tilde"][np.ix_(ids, [2, 3])] = rows[:, 0:2]
        s["bus_w"][j] = rows[:, 2]
        s["bus_th"][j] = rows[:, 3]
        s["br_lam"][np.ix_(ids, [2, 3, 5, 7])] = rows[:, 4:8]


def _admm_net():
    from paper_2106_14995_gb300 import synth
    return synth.network(240, 60, 80, rng=np.random.default_rng(21))


def _admm_worker(rank, world, port, out_dir, iters):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    net = _admm_net()
    part = xdist.partition_buses(net, world)
    plan = xdist.AdmmHaloPlan(net, part, rank)
    eng = _OracleEngine(net)
    hist = np.array([xdist.partitioned_admm_step(eng, plan) for _ in range(iters)])
    np.save(os.path.join(out_dir, f"h{rank}.npy"), hist)
    for k, v in eng.a.arrays.items():
        np.save(os.path.join(out_dir, f"{k}{rank}.npy"), v)
    np.save(os.path.join(out_dir, f"sent{rank}.npy"), np.array([plan.doubles_per_iteration()]))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_covers_buses_balances_cost_and_cuts_few_branches():
    from paper_2106_14995_gb300 import synth
    net = synth.network(10000, 3000, 3000, seed_index=2)
    f, t = net["br_from"], net["br_to"]
    rng = np.random.default_rng(3)
    iters = rng.integers(1, 18, len(f)).astype(float)  # previous TRON iteration counts
    for nparts in (2, 8):
        part = xdist.partition_buses(net, nparts, iters)
        assert part.min() == 0 and part.max() == nparts - 1
        cost = xdist.bus_costs(net, iters)
        per = np.array([cost[part == r].sum() for r in range(nparts)])
        assert per.max() <= cost.sum() / nparts + cost.max()
        plans = [xdist.AdmmHaloPlan(net, part, r) for r in range(nparts)]
        # every component has exactly one owner
        for key in ("own_bus", "own_gen", "own_branch"):
            np.testing.assert_array_equal(sum(getattr(p, key).astype(int) for p in plans), 1)
        cut = part[f] != part[t]
        assert plans[0].cut_branches == cut.sum()
        # the two directions of every exchange name the same branches
        for p in plans:
            for q, ids in p.send_values.items():
                np.testing.assert_array_equal(plans[q].recv_values[p.rank], ids)
        # depth-first blocks cut far fewer branches than an equal-size random split
        rand = rng.permutation(np.repeat(np.arange(nparts), -(-net["nbus"] // nparts))
                               [:net["nbus"]])
        assert cut.sum() < 0.5 * (rand[f] != rand[t]).sum()


def test_partitioned_admm_on_two_gloo_ranks_equals_the_undivided_iteration(tmp_path):
    import oracle
    world, iters = 2, 40
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_admm_worker, args=(r, world, port, str(tmp_path), iters))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    net = _admm_net()
    ref = oracle.Admm(net)
    hp, hd = ref.run(iters)
    part = xdist.partition_buses(net, world)
    assert (part[net["br_from"]] != part[net["br_to"]]).any()  # some branches are cut
    for r in range(world):
        h = np.load(tmp_path / f"h{r}.npy")
        # the residual sums add in another order: equal to rounding
        np.testing.assert_allclose(h[:, 0], hp, rtol=1e-12)
        np.testing.assert_allclose(h[:, 1], hd, rtol=1e-12)
    # recombined from the owners, every iterate equals the undivided run's bit for bit
    f, t, g = net["br_from"], net["br_to"], net["gen_bus"]
    own = {k: {} for k in ("branch", "bus", "gen")}
    for r in range(world):
        own["branch"][r] = part[f] == r
        own["bus"][r] = part == r
        own["gen"][r] = part[g] == r
    for key, kind in (("br_x", "branch"), ("br_delta", "branch"), ("br_val", "branch"),
                      ("bus_w", "bus"), ("bus_th", "bus"), ("gen_pq", "gen"),
                      ("gen_lam", "gen"), ("gen_tilde", "gen")):
        got = np.zeros_like(ref.arrays[key])
        for r in range(world):
            got[own[kind][r]] = np.load(tmp_path / f"{key}{r}.npy")[own[kind][r]]
        np.testing.assert_array_equal(got, ref.arrays[key], err_msg=key)
    # multipliers and flow copies: the from end's pairs live with the branch owner, the
    # to end's with the to-bus owner (and come back to the branch owner each iteration)
    for key in ("br_lam", "br_tilde"):
        np.testing.assert_array_equal(np.load(tmp_path / f"{key}0.npy")[own["branch"][0]],
                                      ref.arrays[key][own["branch"][0]], err_msg=key)
    sent = sum(int(np.load(tmp_path / f"sent{r}.npy")[0]) for r in range(world))
    cut = int((part[f] != part[t]).sum())
    assert sent == 12 * cut
