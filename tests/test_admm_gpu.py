"""GPU component ADMM (Sec. 6.1) against the oracle, checkpoint/resume, and the resident
pool's independence of its co-residents.  Tolerance on residual trajectories: 1e-6
relative (the stated target)."""
import numpy as np
import pytest

import oracle
from paper_2106_14995_gb300 import synth
from paper_2106_14995_gb300.admm import Admm, AdmmPool
from paper_2106_14995_gb300.tron import options

pytestmark = pytest.mark.gpu


def small_net(nb, seed):
    return synth.network(nb, nchord=max(1, nb // 4), ngen=max(1, nb // 3),
                         rng=np.random.default_rng(seed))


@pytest.mark.parametrize("group", [1, 2, 4])
def test_admm_residual_trajectory_matches_oracle(group):
    # group: lanes per branch problem in the branch launch (4 is the default)
    net = small_net(60, 3)
    K = 12
    g = Admm(net, opts=options(group=group))
    g.step(K)
    hp_g, hd_g = g.history(0, K)
    o = oracle.Admm(net)
    hp_o, hd_o = o.run(K, nthreads=4)
    np.testing.assert_allclose(hp_g, hp_o, rtol=1e-6, atol=0)
    np.testing.assert_allclose(hd_g, hd_o, rtol=1e-6, atol=0)
    s = g.get_state()
    assert s["iteration"] == K
    for k in ("br_x", "br_val", "br_tilde", "bus_w", "bus_th", "gen_pq", "gen_tilde"):
        np.testing.assert_allclose(s[k], o.arrays[k], rtol=1e-6, atol=1e-8, err_msg=k)
    np.testing.assert_allclose(s["br_lam"], o.arrays["br_lam"], rtol=1e-6, atol=1e-5)
    np.testing.assert_allclose(s["gen_lam"], o.arrays["gen_lam"], rtol=1e-6, atol=1e-5)
    g.close()


@pytest.mark.parametrize("group", [1, 2, 4])
@pytest.mark.parametrize("nb,seed,K", [(120, 11, 600), (200, 12, 400)])
def test_admm_long_trajectory_matches_oracle(group, nb, seed, K):
    # past the start-up: the branch solves that need the most TRON iterations (and the
    # Cholesky shifts and boundary steps of the PCG) come after the first hundred ADMM
    # iterations; the residual histories must stay within 1e-6 relative of the
    # oracle's at every iteration, not only at the first few
    net = small_net(nb, seed)
    g = Admm(net, opts=options(group=group))
    g.step(K)
    hp_g, hd_g = g.history(0, K)
    o = oracle.Admm(net)
    hp_o, hd_o = o.run(K, nthreads=8)
    np.testing.assert_allclose(hp_g, hp_o, rtol=1e-6, atol=0)
    np.testing.assert_allclose(hd_g, hd_o, rtol=1e-6, atol=0)
    s = g.get_state()
    for k in ("br_x", "br_val", "br_tilde", "bus_w", "bus_th", "gen_pq", "gen_tilde"):
        np.testing.assert_allclose(s[k], o.arrays[k], rtol=1e-6, atol=1e-8, err_msg=k)
    g.close()


@pytest.mark.parametrize("group", [1, 4])
def test_admm_with_the_hessian_norm_cauchy_option_matches_oracle(group):
    net = small_net(120, 11)
    K = 300
    g = Admm(net, opts=options(group=group, cauchy_norm=1))
    g.step(K)
    hp_g, hd_g = g.history(0, K)
    g.close()
    hp_o, hd_o = oracle.Admm(net).run(K, opts=oracle.default_opts(cauchy_norm=1), nthreads=8)
    np.testing.assert_allclose(hp_g, hp_o, rtol=1e-6, atol=0)
    np.testing.assert_allclose(hd_g, hd_o, rtol=1e-6, atol=0)


@pytest.mark.parametrize("split", [1, -1])
def test_one_lane_split_continuation_matches_oracle(split):
    # one lane per branch problem; split 1: every solve still running after one TRON
    # iteration is finished on four lanes by the third launch (so nearly every solve
    # resumes from x, delta, its iteration count and Cauchy step), -1: never split
    net = small_net(120, 11)
    K = 400
    g = Admm(net, opts=options(group=1, split_outer=split))
    assert g.branch_group == 1
    assert g.launches_per_iteration == (3 if split > 0 else 2)
    g.step(K)
    hp_g, hd_g = g.history(0, K)
    s = g.get_state()
    counts = g.branch_status_counts()
    g.close()
    # every solve ended with a reported status (none left paused)
    assert counts.sum() == len(net["br_from"])
    o = oracle.Admm(net)
    hp_o, hd_o = o.run(K, nthreads=8)
    np.testing.assert_allclose(hp_g, hp_o, rtol=1e-6, atol=0)
    np.testing.assert_allclose(hd_g, hd_o, rtol=1e-6, atol=0)
    for k in ("br_x", "br_val", "br_tilde", "bus_w", "bus_th", "gen_pq"):
        np.testing.assert_allclose(s[k], o.arrays[k], rtol=1e-6, atol=1e-8, err_msg=k)


def test_launches_per_iteration_follow_the_branch_mapping():
    net = small_net(60, 3)
    for grp, split, want in ((4, 0, 2), (4, 2, 2), (1, 0, 2), (1, 2, 3), (1, -1, 2)):
        a = Admm(net, opts=options(group=grp, split_outer=split))
        assert a.launches_per_iteration == want, (grp, split)
        a.close()


def test_admm_light_load_rho10_converges_where_the_oracle_does():
    # an instance of the serving benchmark's convergent request set (515 buses, a tenth
    # of the stated load, rho 10): the GPU trajectory follows the oracle's through
    # convergence, and both first reach primal and dual <= 1e-4 at the same iteration
    specs = synth.serving_stream(duration_s=0.5, rate_hz=200.0, seed_index=5, bus_lo=500,
                                 bus_hi=2000, load_lo=0.08, load_hi=0.12)
    spec = specs[78]
    assert spec["nbus"] == 515
    net = synth.instance_network(spec)
    K = 1200
    g = Admm(net, rho=10.0)
    g.step(K)
    hp_g, hd_g = g.history(0, K)
    g.close()
    hp_o, hd_o = oracle.Admm(net, rho=10.0).run(K, nthreads=8)
    np.testing.assert_allclose(hp_g, hp_o, rtol=1e-6, atol=0)
    np.testing.assert_allclose(hd_g, hd_o, rtol=1e-6, atol=0)
    first_g = np.nonzero((hp_g <= 1e-4) & (hd_g <= 1e-4))[0]
    first_o = np.nonzero((hp_o <= 1e-4) & (hd_o <= 1e-4))[0]
    assert first_o.size and first_g.size and first_g[0] == first_o[0]


def test_admm_2000_bus_trajectory_matches_oracle():
    net = small_net(2000, 13)
    K = 150
    for group in (1, 4):
        g = Admm(net, opts=options(group=group))
        g.step(K)
        hp_g, hd_g = g.history(0, K)
        if group == 1:
            o = oracle.Admm(net)
            hp_o, hd_o = o.run(K, nthreads=8)
        np.testing.assert_allclose(hp_g, hp_o, rtol=1e-6, atol=0)
        np.testing.assert_allclose(hd_g, hd_o, rtol=1e-6, atol=0)
        s = g.get_state()
        np.testing.assert_allclose(s["br_x"], o.arrays["br_x"], rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(s["bus_w"], o.arrays["bus_w"], rtol=1e-6, atol=1e-8)
        g.close()


def test_branch_group_default_follows_branch_slots_per_sm():
    # four lanes per branch problem while the pool holds <= 24 branch slots per SM
    # sub-partition, else one; an explicit options.group wins; the default run equals
    # the explicit run of the same mapping bit for bit
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    net = small_net(60, 3)
    a = Admm(net)
    b = Admm(net, opts=options(group=4))
    assert a.branch_group == 4 and b.branch_group == 4
    a.step(5)
    b.step(5)
    np.testing.assert_array_equal(a.history(0, 5)[0], b.history(0, 5)[0])
    np.testing.assert_array_equal(a.get_state()["br_x"], b.get_state()["br_x"])
    a.close()
    b.close()
    big = 24 * 4 * nsm + 128
    p = AdmmPool(1000, big, 1000, 2)
    assert p.branch_group == 1
    p.close()
    p = AdmmPool(1000, big, 1000, 2, opts=options(group=4))
    assert p.branch_group == 4
    p.close()
    p = AdmmPool(1000, 24 * 4 * nsm, 1000, 2)
    assert p.branch_group == 4
    p.close()


def test_admm_larger_network_tracks_oracle():
    net = small_net(400, 4)
    K = 6
    g = Admm(net)
    g.step(K)
    hp_g, hd_g = g.history(0, K)
    hp_o, hd_o = oracle.Admm(net).run(K, nthreads=8)
    np.testing.assert_allclose(hp_g, hp_o, rtol=1e-6)
    np.testing.assert_allclose(hd_g, hd_o, rtol=1e-6)
    counts = g.branch_status_counts()
    assert counts.sum() == len(net["br_from"])
    g.close()


def test_admm_step_returns_last_residuals_and_counts_iterations():
    net = small_net(30, 5)
    g = Admm(net)
    pr, du = g.step(9)
    assert g.iterations == 9
    hp, hd = g.history(8, 1)
    assert pr == hp[0] and du == hd[0]
    pr2, du2 = g.step(8)  # one full replayed graph chunk
    assert g.iterations == 17
    assert np.isfinite(pr2) and np.isfinite(du2)
    g.close()


def test_admm_checkpoint_resume_is_bitwise():
    net = small_net(80, 6)
    g = Admm(net)
    g.step(7)
    saved = g.get_state()
    g.step(5)
    ref = g.get_state()
    ref_hist = g.history(7, 5)
    g2 = Admm(net)
    g2.set_state(saved)
    assert g2.iterations == 7
    g2.step(5)
    got = g2.get_state()
    for k, v in ref.items():
        np.testing.assert_array_equal(got[k], v, err_msg=k)
    h = g2.history(7, 5)
    np.testing.assert_array_equal(h[0], ref_hist[0])
    np.testing.assert_array_equal(h[1], ref_hist[1])
    g.close()
    g2.close()


def _alone(net, iters, group=0, split=0):
    p = AdmmPool(len(net["bus_pd"]) + 256, len(net["br_from"]) + 256,
                 len(net["gen_bus"]) + 256, 1, opts=options(group=group, split_outer=split))
    i = p.add(net)
    p.step(iters)
    st = p.get_state(i)
    hist = p.history(i, 0, iters)
    p.close()
    return st, hist


@pytest.mark.parametrize("group,split", [(4, 0), (2, 0), (1, 0), (1, 1)])
def test_pool_results_identical_alone_and_in_the_mix(group, split):
    # every branch mapping: an instance's results do not depend on its co-residents --
    # with split 1 also when nearly every solve is finished by the tail launch, whose
    # list of paused solves is filled in whatever order their warps reach it
    nets = [small_net(40, 11), small_net(130, 12), small_net(25, 13), small_net(70, 14)]
    pool = AdmmPool(4000, 4000, 2000, 4, opts=options(group=group, split_outer=split))
    assert pool.branch_group == group
    assert pool.launches_per_iteration == (3 if split > 0 else 2)
    a = pool.add(nets[0])
    pool.step(5)
    b = pool.add(nets[1])          # admitted while a is running
    pool.step(3)
    c = pool.add(nets[2])
    pool.step(9)                   # a: 17, b: 12, c: 9 iterations
    it, pr, du = pool.residuals()
    assert it[a] == 17 and it[b] == 12 and it[c] == 9
    sa, sb, sc = pool.get_state(a), pool.get_state(b), pool.get_state(c)
    pool.remove(b)                 # free b's slots, admit d into them
    d = pool.add(nets[3])
    pool.step(4)                   # a: 21, c: 13, d: 4
    sa2, sd = pool.get_state(a), pool.get_state(d)
    for net, st, iters in ((nets[0], sa, 17), (nets[1], sb, 12), (nets[2], sc, 9),
                           (nets[0], sa2, 21), (nets[3], sd, 4)):
        ref, _ = _alone(net, iters, group, split)
        for k in ref:
            np.testing.assert_array_equal(st[k], ref[k], err_msg=k)
    assert pool.live == 3
    pool.close()


def test_pool_rejects_when_full_and_reuses_slots():
    pool = AdmmPool(250, 400, 200, 2)  # 256 bus slots after alignment
    n1 = small_net(100, 21)
    n2 = small_net(250, 22)  # does not fit next to n1 (bus slots are 128-aligned)
    i1 = pool.add(n1)
    assert i1 is not None
    assert pool.add(n2) is None
    pool.remove(i1)
    assert pool.add(n2) is not None
    pool.close()


def test_serving_loop_admits_waits_retires_and_matches_alone_runs():
    from paper_2106_14995_gb300.serving import AdmmServer, serial_plain, summarize
    rng = np.random.default_rng(31)
    reqs = []
    for k in range(7):
        nb = int(rng.integers(20, 160))
        reqs.append(dict(id=k, t=0.0, net=small_net(nb, 100 + k)))
    # all arrive at once, with room for at most three instances: the later ones are
    # admitted only as earlier ones retire (decided by capacity, not by timing)
    server = AdmmServer(cap_bus=384, cap_branch=512, cap_gen=256, cap_instances=3, chunk=4,
                        tol=1e-4, max_iters=12)
    recs = server.run(reqs, keep_state=True)
    server.close()
    assert sorted(r["id"] for r in recs) == list(range(7))
    first_done = min(r["finished"] for r in recs)
    waited = [r for r in recs if r["admitted"] >= first_done]
    assert len(waited) >= 7 - 3  # admitted only after a retirement freed slots
    for r in recs:  # never more than three live at once
        live = sum(1 for q in recs if q["admitted"] <= r["admitted"] < q["finished"])
        assert live <= 3
    for r in recs:
        assert r["iterations"] == 12 or r["converged"]
        alone = Admm(reqs[r["id"]]["net"])
        alone.step(r["iterations"])
        ref = alone.get_state()
        alone.close()
        for k in ref:
            np.testing.assert_array_equal(r["state"][k], ref[k], err_msg=f"{r['id']} {k}")
    s = summarize(recs)
    assert s["instances"] == 7 and s["p99_s"] >= s["p50_s"] > 0
    serial = serial_plain(reqs, chunk=4, max_iters=12)
    assert [x["iterations"] for x in sorted(serial, key=lambda x: x["id"])] == \
        [x["iterations"] for x in sorted(recs, key=lambda x: x["id"])]


def test_admm_full_size_network_tracks_oracle():
    # the benchmark's network (10,000 buses, 13,000 branches, 3,000 generators)
    net = synth.network(10000, 3000, 3000, seed_index=2)
    o = oracle.Admm(net)
    hp, hd = o.run(6, nthreads=8)
    g = Admm(net)
    res = np.array([g.step(1) for _ in range(6)])
    np.testing.assert_allclose(res[:, 0], hp, rtol=1e-6)
    np.testing.assert_allclose(res[:, 1], hd, rtol=1e-6)
    s = g.get_state()
    rng = np.random.default_rng(0)
    ks = rng.choice(13000, 500, replace=False)
    np.testing.assert_allclose(s["br_x"][ks], o.arrays["br_x"][ks], rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(s["bus_w"], o.arrays["bus_w"], rtol=1e-6, atol=1e-8)
    np.testing.assert_allclose(s["gen_pq"], o.arrays["gen_pq"], rtol=1e-6, atol=1e-8)
    g.close()


def _edge_network():
    # 5 buses: bus 3 has no branch (a generator and a load only), bus 4 carries two
    # generators, bus 2 has neither generator nor load; branches 0-1, 1-2, 2-4, 4-0
    rng = np.random.default_rng(60)
    br_from = np.array([0, 1, 2, 4], dtype=np.int32)
    br_to = np.array([1, 2, 4, 0], dtype=np.int32)
    r, x, bc, smax = synth.random_lines(rng, 4)
    return dict(nbus=5, br_from=br_from, br_to=br_to,
                br_coef=synth.line_coefficients(r, x, bc), br_smax2=smax * smax,
                gen_bus=np.array([3, 4, 4, 1], dtype=np.int32),
                gen_c2=np.array([0.01, 0.02, 0.03, 0.015]),
                gen_c1=np.array([10.0, 20.0, 15.0, 12.0]),
                gen_pmin=np.zeros(4), gen_pmax=np.array([1.0, 0.8, 0.6, 1.2]),
                gen_qmin=np.full(4, -0.5), gen_qmax=np.full(4, 0.5),
                bus_pd=np.array([0.3, 0.2, 0.0, 0.4, 0.5]),
                bus_qd=np.array([0.05, 0.1, 0.0, 0.1, 0.0]),
                bus_gsh=np.zeros(5), bus_bsh=np.zeros(5))


def test_admm_edge_network_isolated_and_multi_generator_buses():
    net = _edge_network()
    o = oracle.Admm(net)
    hp, hd = o.run(25)
    g = Admm(net)
    res = np.array([g.step(1) for _ in range(25)])
    np.testing.assert_allclose(res[:, 0], hp, rtol=1e-6)
    np.testing.assert_allclose(res[:, 1], hd, rtol=1e-6)
    s = g.get_state()
    for k in ("gen_pq", "gen_lam", "bus_w", "bus_th", "br_x", "br_lam"):
        np.testing.assert_allclose(s[k], o.arrays[k], rtol=1e-6, atol=1e-8, err_msg=k)
    # the isolated bus keeps its voltage (no branch copies to average)
    assert s["bus_w"][3] == 1.0 and s["bus_th"][3] == 0.0
    g.close()


@pytest.mark.parametrize("group", [4, 2, 1])
def test_pool_instances_with_their_own_penalties_and_boxes(group):
    # instances that differ in rho, the line penalty and the voltage box share every
    # launch; each equals its own run alone bit for bit and follows the oracle's
    # trajectory for its parameters
    cases = [(small_net(40, 21), dict(rho=10.0, rho_line=10.0, vmin=0.9, vmax=1.1)),
             (small_net(60, 22), dict(rho=400.0, rho_line=1000.0, vmin=0.95, vmax=1.05)),
             (small_net(30, 23), dict(rho=1000.0, rho_line=200.0, vmin=0.85, vmax=1.15))]
    K = 60
    pool = AdmmPool(2000, 2000, 1000, 3, opts=options(group=group))
    ids = [pool.add(net, **kw) for net, kw in cases]
    pool.step(K)
    for i, (net, kw) in zip(ids, cases):
        st = pool.get_state(i)
        hp, hd = pool.history(i, 0, K)
        solo = AdmmPool(2000, 2000, 1000, 1, opts=options(group=group))
        j = solo.add(net, **kw)
        solo.step(K)
        ref = solo.get_state(j)
        for k in ref:
            np.testing.assert_array_equal(st[k], ref[k], err_msg=k)
        solo.close()
        hp_o, hd_o = oracle.Admm(net, **kw).run(K, nthreads=4)
        np.testing.assert_allclose(hp, hp_o, rtol=1e-6, atol=0)
        np.testing.assert_allclose(hd, hd_o, rtol=1e-6, atol=0)
    pool.close()
