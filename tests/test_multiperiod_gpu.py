"""GPU parity of the multi-period pieces against the oracle: the generator-chain
objective (TRON_OBJ_GEN_RAMP) solved by the batched TRON kernel, and the multi-period
ADMM (admm_mp_*).

Tolerances as elsewhere: the chain problems are strictly convex, so x within 1e-6 and
f within 1e-8 relative of the oracle; ADMM residual trajectories within 1e-6 relative."""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_14995_gb300 import native, synth
from paper_2106_14995_gb300.admm import Admm, AdmmMultiPeriod
from paper_2106_14995_gb300.tron import TronBatch, options

pytestmark = pytest.mark.gpu


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _gpu_batch(d, **opt):
    B = d["delta0"].shape[0]
    tb = TronBatch(4, B, n=d["n"], opts=options(**opt))
    out = tb.solve(_t(d["params"]), _t(d["l"]), _t(d["u"]), _t(d["x0"]), _t(d["delta0"]))
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    tb.close()
    return res


@pytest.mark.parametrize("T", [24, 12, 5, 32, 1])
def test_genramp_batch_parity(T):
    d = synth.genramp_batch(301, T, seed_index=40 + T)
    g = _gpu_batch(d)
    r = oracle.tron_batch(4, d["params"], d["l"], d["u"], d["x0"], d["delta0"], nthreads=8)
    assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
    assert np.all(r["status"] == oracle.CONVERGED)
    assert np.all(g["pg"] <= 1e-6)
    np.testing.assert_allclose(g["x"], r["x"], rtol=0, atol=1e-6)
    rel = np.abs(g["f"] - r["f"]) / np.maximum(1.0, np.abs(r["f"]))
    assert rel.max() <= 1e-8
    g2 = _gpu_batch(d, schedule=native.TRON_SCHED_PERSISTENT)
    for k in ("x", "f", "iters", "status"):
        np.testing.assert_array_equal(g2[k], g[k])


def test_genramp_without_binding_ramps_is_the_closed_form():
    d = synth.genramp_batch(200, 24, seed_index=48)
    d["params"][:, 4] = 1e6
    g = _gpu_batch(d)
    rec = d["params"]
    c2, c1, rho = rec[:, 0:1], rec[:, 1:2], rec[:, 2:3]
    lam, tgt = rec[:, 8:32], rec[:, 32:56]
    closed = np.clip((rho * tgt - lam - c1) / (2 * c2 + rho), d["l"], d["u"])
    np.testing.assert_allclose(g["x"], closed, rtol=0, atol=1e-9)


def _small_net(nbus, seed):
    return synth.network(nbus, nchord=max(1, nbus // 4), ngen=max(1, nbus // 3),
                         rng=np.random.default_rng(seed))


def test_multiperiod_admm_matches_oracle():
    net = _small_net(40, 50)
    scale = synth.load_profile(4)
    kw = dict(ramp=0.02, rho_ramp=1e4)
    o = oracle.MultiPeriodAdmm(net, scale, **kw)
    hp, hd = o.run(15, nthreads=8)
    g = AdmmMultiPeriod(net, scale, **kw)
    res = np.array([g.step(1) for _ in range(15)])
    np.testing.assert_allclose(res[:, 0], hp, rtol=1e-6)
    np.testing.assert_allclose(res[:, 1], hd, rtol=1e-6)
    for t in range(4):
        s = g.get_state(t)
        assert s["iteration"] == 15
        for k in ("gen_pq", "bus_w", "bus_th", "br_x"):
            np.testing.assert_allclose(s[k], o.state(t)[k], rtol=1e-6, atol=1e-8, err_msg=k)
    p = np.array([g.get_state(t)["gen_pq"][:, 0] for t in range(4)])
    assert np.abs(np.diff(p, axis=0)).max() < 0.05  # the ramps hold, up to the penalty
    assert g.gen_status_counts()[native.TRON_CONVERGED] == len(net["gen_bus"])
    g.close()


def test_multiperiod_one_lane_split_matches_oracle():
    # one lane per branch with every solve still running after one TRON iteration
    # finished on four lanes, and the generator chains on the side stream beside them
    net = _small_net(40, 50)
    scale = synth.load_profile(4)
    kw = dict(ramp=0.02, rho_ramp=1e4)
    o = oracle.MultiPeriodAdmm(net, scale, **kw)
    hp, hd = o.run(40, nthreads=8)
    g = AdmmMultiPeriod(net, scale, opts=options(group=1, split_outer=1), **kw)
    assert g.launches_per_iteration == 6
    res = np.array([g.step(1) for _ in range(40)])
    np.testing.assert_allclose(res[:, 0], hp, rtol=1e-6)
    np.testing.assert_allclose(res[:, 1], hd, rtol=1e-6)
    for t in range(4):
        s = g.get_state(t)
        for k in ("gen_pq", "bus_w", "bus_th", "br_x"):
            np.testing.assert_allclose(s[k], o.state(t)[k], rtol=1e-6, atol=1e-8, err_msg=k)
    g.close()


def test_multiperiod_without_binding_ramps_equals_single_period_runs():
    net = _small_net(50, 51)
    scale = [0.9, 1.0, 1.1]
    g = AdmmMultiPeriod(net, scale, ramp=1e6)
    g.step(10)
    for t, s in enumerate(scale):
        a = Admm(dict(net, bus_pd=net["bus_pd"] * s, bus_qd=net["bus_qd"] * s))
        a.step(10)
        ref = a.get_state()
        got = g.get_state(t)
        for k in ("gen_pq", "gen_lam", "bus_w", "br_x", "br_lam"):
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-9, atol=1e-9, err_msg=k)
        a.close()
    g.close()


def test_zero_ramp_penalty_gives_independent_scenarios():
    # independent load scenarios of one network as one multi-period instance: with
    # rho_ramp = 0 each generator chain falls apart into its periods' own problems, so the
    # scenarios equal separate single-period runs -- here with ramp limits that a penalty
    # would make bind, and load factors drawn as the serving requests' are
    net = _small_net(60, 53)
    scale = np.random.default_rng(54).uniform(0.8, 1.2, 8)
    g = AdmmMultiPeriod(net, scale, ramp=0.01, rho_ramp=0.0)
    g.step(10)
    for t, s in enumerate(scale):
        a = Admm(dict(net, bus_pd=net["bus_pd"] * s, bus_qd=net["bus_qd"] * s))
        a.step(10)
        ref = a.get_state()
        got = g.get_state(t)
        for k in ("gen_pq", "gen_lam", "bus_w", "br_x", "br_lam"):
            np.testing.assert_allclose(got[k], ref[k], rtol=1e-9, atol=1e-9, err_msg=k)
        a.close()
    g.close()


def test_multiperiod_rejects_bad_arguments():
    net = _small_net(20, 52)
    with pytest.raises(native.TronError, match="EINVAL"):
        AdmmMultiPeriod(net, np.ones(33), ramp=0.1)
    with pytest.raises(native.TronError, match="EINVAL"):
        AdmmMultiPeriod(net, np.ones(4), ramp=-0.1)
    with pytest.raises(native.TronError, match="EINVAL"):
        AdmmMultiPeriod(net, [1.0, 0.0], ramp=0.1)


def test_multiperiod_benchmark_size_tracks_oracle():
    # the benchmark's workload: 24 periods x (2,000 buses, 2,600 branches, 600 generators)
    net = synth.network(2000, 600, 600, seed_index=9)
    scale = synth.load_profile(24)
    kw = dict(ramp=0.05 * net["gen_pmax"], rho_ramp=1e4)
    o = oracle.MultiPeriodAdmm(net, scale, **kw)
    hp, hd = o.run(3, nthreads=8)
    g = AdmmMultiPeriod(net, scale, **kw)
    res = np.array([g.step(1) for _ in range(3)])
    np.testing.assert_allclose(res[:, 0], hp, rtol=1e-6)
    np.testing.assert_allclose(res[:, 1], hd, rtol=1e-6)
    for t in (0, 11, 23):
        np.testing.assert_allclose(g.get_state(t)["gen_pq"], o.state(t)["gen_pq"], rtol=1e-6,
                                   atol=1e-8)
    g.close()


@pytest.mark.parametrize("T", [1, 32])
def test_multiperiod_edge_period_counts_match_oracle(T):
    # one period (the chains reduce to single generators) and the most periods a chain
    # holds (32, one per lane of a warp)
    net = _small_net(30, 53)
    scale = synth.load_profile(T)
    kw = dict(ramp=0.03, rho_ramp=1e4)
    hp, hd = oracle.MultiPeriodAdmm(net, scale, **kw).run(12, nthreads=8)
    g = AdmmMultiPeriod(net, scale, **kw)
    res = np.array([g.step(1) for _ in range(12)])
    np.testing.assert_allclose(res[:, 0], hp, rtol=1e-6)
    np.testing.assert_allclose(res[:, 1], hd, rtol=1e-6)
    g.close()
