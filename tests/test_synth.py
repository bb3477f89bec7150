"""The seeded input generators against the recipes they state (CPU only): determinism,
ranges and layouts of the branch and dense records, the network's structure (spanning
tree plus distinct chords, generators on distinct buses), the uneven size mix, the load
profile, the serving stream and the generator-chain records."""
import math

import numpy as np

from paper_2106_14995_gb300 import synth


def test_same_seed_same_inputs():
    a, b = synth.branch_batch(64, seed_index=3), synth.branch_batch(64, seed_index=3)
    for k in ("params", "l", "u", "x0", "delta0"):
        np.testing.assert_array_equal(a[k], b[k])
    c = synth.branch_batch(64, seed_index=4)
    assert not np.array_equal(a["params"], c["params"])
    n1, n2 = synth.network(300, 60, 50, seed_index=7), synth.network(300, 60, 50, seed_index=7)
    for k in ("br_from", "br_to", "br_coef", "gen_bus", "bus_pd"):
        np.testing.assert_array_equal(n1[k], n2[k])


def test_branch_records_follow_the_recipe():
    d = synth.branch_batch(4000, seed_index=0)
    rec = d["params"]
    assert rec.shape == (4000, synth.BRANCH_RECORD)
    lam, tgt = rec[:, 8:16], rec[:, 16:24]
    assert abs(lam.mean()) < 0.05 and abs(lam.std() - 1.0) < 0.05
    assert abs(tgt.mean()) < 0.03 and abs(tgt.std() - 0.5) < 0.03
    assert np.all(rec[:, 24:32] == 400.0) and np.all(rec[:, 33] == 400.0)
    assert np.all((rec[:, 32] >= 0.25) & (rec[:, 32] <= 4.0))   # smax in [0.5, 2]
    assert np.all(rec[:, 34:] == 0.0)
    np.testing.assert_array_equal(d["l"][0], [0.9, 0.9, -2 * math.pi, -2 * math.pi])
    np.testing.assert_array_equal(d["u"][0], [1.1, 1.1, 2 * math.pi, 2 * math.pi])
    np.testing.assert_array_equal(d["x0"][0], [1.0, 1.0, 0.0, 0.0])
    # series admittance 1 / (r + jx), r in [0.001, 0.05], x in [0.01, 0.3]: the
    # conductance g_ij = r / (r^2 + x^2) and b_ij = x / (r^2 + x^2) are positive, and
    # r^2 + x^2 >= 2 r x bounds g_ij by 1 / (2 x) <= 50
    g, b = rec[:, 2], rec[:, 3]
    assert np.all(g > 0) and np.all(g <= 50.0) and np.all(b > 0)


def test_line_coefficients_are_the_pi_model():
    r, x, bc = np.array([0.02]), np.array([0.1]), np.array([0.04])
    c = synth.line_coefficients(r, x, bc)[0]
    y = 1.0 / complex(0.02, 0.1)
    # the shunt-side coefficients of both ends are equal, the series ones too
    assert c[0] == c[4] and c[1] == c[5] and c[2] == c[6] and c[3] == c[7]
    assert math.isclose(c[2], y.real, rel_tol=1e-12)
    assert math.isclose(c[3], -y.imag, rel_tol=1e-12)
    assert math.isclose(c[1], -(y.imag + 0.02), rel_tol=1e-12)


def test_dense_records_follow_the_recipe():
    d = synth.dense_batch(200, 16, seed_index=1)
    n = 16
    Q = d["params"][:, : n * n].reshape(-1, n, n)
    np.testing.assert_array_equal(Q, np.transpose(Q, (0, 2, 1)))
    ev = np.linalg.eigvalsh(Q)
    assert ev.min() >= 1.0 - 1e-9 and ev.max() <= 1e3 * (1 + 1e-9)
    c = d["params"][:, n * n: n * n + n]
    assert abs(c.std() - 4.0) < 0.2
    assert np.all(d["params"][:, n * n + n:] == 0.1)
    assert np.all((d["l"] >= -2.0) & (d["l"] <= -0.5))
    assert np.all((d["u"] >= 0.5) & (d["u"] <= 2.0))
    assert np.all(d["x0"] == 0.0) and np.all(d["delta0"] == 1.0)


def test_network_structure():
    nb, nc, ng = 2000, 600, 500
    net = synth.network(nb, nc, ng, seed_index=5)
    f, t = net["br_from"], net["br_to"]
    assert f.size == nb - 1 + nc
    assert np.all(f != t)
    keys = {(min(a, b), max(a, b)) for a, b in zip(f.tolist(), t.tolist())}
    assert len(keys) == f.size                      # no parallel branches
    # the first nb - 1 branches form a spanning tree: union-find joins every bus
    parent = list(range(nb))

    def root(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    for a, b in zip(f[: nb - 1].tolist(), t[: nb - 1].tolist()):
        ra, rb = root(a), root(b)
        assert ra != rb                              # no cycle inside the tree
        parent[ra] = rb
    assert len({root(a) for a in range(nb)}) == 1
    g = net["gen_bus"]
    assert g.size == ng and np.unique(g).size == ng
    assert np.all((net["gen_c2"] >= 0.001) & (net["gen_c2"] <= 0.05))
    assert np.all((net["gen_c1"] >= 5.0) & (net["gen_c1"] <= 40.0))
    np.testing.assert_array_equal(net["gen_qmax"], 0.5 * net["gen_pmax"])
    np.testing.assert_array_equal(net["gen_qmin"], -0.5 * net["gen_pmax"])
    assert 1.5 < net["gen_pmax"].sum() / net["bus_pd"].sum() < 2.5   # about twice the load
    assert np.all((net["bus_pd"] >= 0) & (net["bus_pd"] <= 1))
    assert np.all((net["bus_qd"] >= -0.2) & (net["bus_qd"] <= 0.5))


def test_uneven_mix_and_layout():
    d = synth.uneven_batch(20000, seed_index=3)
    nv = d["nvec"]
    counts = np.array([(nv == s).sum() for s in synth.UNEVEN_SIZES]) / nv.size
    np.testing.assert_allclose(counts, synth.UNEVEN_PROBS, atol=0.015)
    assert d["params"].size == int((nv.astype(np.int64) ** 2 + 2 * nv).sum())
    assert d["l"].size == d["u"].size == d["x0"].size == int(nv.sum())


def test_load_profile_and_serving_stream():
    s = synth.load_profile(24)
    assert s.argmax() == 12 and math.isclose(s.max(), 1.2)
    assert s.argmin() == 0 and math.isclose(s.min(), 0.8)
    st = synth.serving_stream(duration_s=20.0, rate_hz=200.0)
    assert abs(len(st) / 20.0 - 200.0) < 15.0
    ts = [r["t"] for r in st]
    assert ts == sorted(ts) and ts[-1] <= 20.0
    nb = np.array([r["nbus"] for r in st])
    assert nb.min() >= 500 and nb.max() <= 20000
    # log-uniform: the median bus count near the geometric mean of the range
    assert abs(math.log(np.median(nb)) - 0.5 * (math.log(500) + math.log(20000))) < 0.25


def test_genramp_records():
    d = synth.genramp_batch(500, 24, seed_index=8)
    rec = d["params"]
    pmax = d["u"][:, 0]
    assert rec.shape == (500, 8 + 48)
    assert np.all(rec[:, 2] == 400.0) and np.all(rec[:, 3] == 1e4)
    assert np.all((rec[:, 4] >= 0.02 * pmax - 1e-15) & (rec[:, 4] <= 0.2 * pmax + 1e-15))
    tgt = rec[:, 32:]
    assert np.all((tgt >= 0) & (tgt <= pmax[:, None]))
    np.testing.assert_array_equal(d["x0"], tgt)
