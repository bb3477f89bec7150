"""GPU parity of batched TRON against the CPU oracle, through the C ABI.

Tolerances (from the stated accuracy targets): projected-gradient max-norm <= 1e-6 for
every converged problem; on convex problems ||x_gpu - x_oracle||_inf <= 1e-6 and
relative objective difference <= 1e-8; on nonconvex problems (branch, hs45) x within
1e-6 where both runs took the same path, otherwise both must be KKT points.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_14995_gb300 import native, synth
from paper_2106_14995_gb300.tron import TronBatch, options

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=DEV)


def gpu_solve(d, n=None, n_list=None, **opt):
    B = d["delta0"].shape[0]
    o = options(**opt)
    tb = TronBatch(d["kind"], B, n=n if n_list is None else None, n_list=n_list, opts=o)
    params = _t(d["params"]) if np.size(d["params"]) else None
    x = _t(d["x0"])
    delta = _t(d["delta0"])
    out = tb.solve(params, _t(d["l"]), _t(d["u"]), x, delta)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["launches"] = tb.last_launches
    tb.close()
    return res


def oracle_solve(d, n_list=None, **opt):
    return oracle.tron_batch(d["kind"], d["params"] if np.size(d["params"]) else None, d["l"],
                             d["u"], d["x0"], d["delta0"], n=n_list,
                             opts=oracle.default_opts(**opt), nthreads=8)


def assert_convex_parity(g, r, l, u):
    assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
    assert np.all(r["status"] == oracle.CONVERGED)
    assert np.all(g["pg"] <= 1e-6)
    np.testing.assert_allclose(g["x"], r["x"], rtol=0, atol=1e-6)
    rel = np.abs(g["f"] - r["f"]) / np.maximum(1.0, np.abs(r["f"]))
    assert rel.max() <= 1e-8, rel.max()
    assert np.all(g["x"] >= l) and np.all(g["x"] <= u)


def test_dense_n32_parity_ragged():
    # 301 problems of the n = 32 workload: several CTAs and a ragged tail
    d = synth.dense_batch(301, 32, seed_index=1)
    g = gpu_solve(d, n=32)
    r = oracle_solve(d)
    assert g["launches"] == 1
    assert_convex_parity(g, r, d["l"], d["u"])
    # same path: iteration counts agree on (almost) every problem
    assert np.mean(g["iters"] == r["iters"]) >= 0.95


@pytest.mark.parametrize("n", [1, 3, 4, 5, 7, 8, 12, 16, 20, 31, 32, 33, 48, 64, 100, 128])
def test_dense_sizes(n):
    d = synth.dense_batch(97 if n <= 32 else 41, n, seed_index=20 + n)
    g = gpu_solve(d, n=n)
    r = oracle_solve(d)
    assert_convex_parity(g, r, d["l"], d["u"])


@pytest.mark.parametrize("n,group", [(4, 1), (4, 4), (8, 1), (8, 8), (16, 8), (16, 16),
                                     (32, 16), (32, 32)])
def test_dense_group_mappings(n, group):
    d = synth.dense_batch(133, n, seed_index=40 + n)
    g = gpu_solve(d, n=n, group=group)
    r = oracle_solve(d)
    assert_convex_parity(g, r, d["l"], d["u"])


@pytest.mark.parametrize("n,layout", [(32, 2), (32, 4), (64, 2), (64, 4), (128, 4), (100, 4),
                                      (32, 6), (31, 6), (20, 6), (17, 6)])
def test_dense_large_layouts(n, layout):
    # layout option = 1 + bits: 2 = packed factor with Q in shared memory,
    # 4 = packed factor with Q read from global memory, 6 = packed factor with Q as
    # wrapped diagonals (odd and even n, wrapped modulo n inside the n = 32 class)
    d = synth.dense_batch(37, n, seed_index=60 + n)
    g = gpu_solve(d, n=n, layout=layout)
    r = oracle_solve(d)
    assert_convex_parity(g, r, d["l"], d["u"])


@pytest.mark.parametrize("n", [20, 32, 64, 128])
def test_left_and_right_looking_factorizations_agree(n):
    # both forms factor the same matrix (A = Lu D Lu^T); the left-looking one forms the
    # row D Lu^T it updates with, so the factors agree to rounding, not bit for bit
    d = synth.dense_batch(61, n, seed_index=80 + n)
    a = gpu_solve(d, n=n, cholesky=1)
    b = gpu_solve(d, n=n, cholesky=2)
    assert_convex_parity(a, b, d["l"], d["u"])
    assert np.mean(a["iters"] == b["iters"]) >= 0.95
    r = oracle_solve(d)
    assert_convex_parity(a, r, d["l"], d["u"])
    br = synth.branch_batch(96, seed_index=81)
    a = gpu_solve(br, n=4, cholesky=1)
    b = gpu_solve(br, n=4, cholesky=2)
    assert np.all(a["status"] == native.TRON_CONVERGED)
    assert np.all(b["status"] == native.TRON_CONVERGED)
    same = np.all(np.abs(a["x"] - b["x"]) <= 1e-6, axis=1)
    assert same.mean() >= 0.98


def _branch_kkt(rec, x, l, u):
    f, gr, _ = oracle.eval_obj(oracle.OBJ_BRANCH, rec, x)
    return oracle.pgnorm(x, gr, l, u)


@pytest.mark.parametrize("B,group", [(256, 1), (256, 2), (256, 4), (301, 2), (301, 4)])
def test_branch_parity(B, group):
    # group 1: one branch per lane; group 4: one per four lanes (301: a ragged last warp)
    d = synth.branch_batch(B, seed_index=0)
    g = gpu_solve(d, n=4, group=group)
    r = oracle_solve(d)
    assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
    assert np.all(r["status"] == oracle.CONVERGED)
    # the GPU result is a KKT point by the oracle's own gradient
    for p in range(B):
        assert _branch_kkt(d["params"][p], g["x"][p], d["l"][p], d["u"][p]) <= 1e-6 * 1.01
    same = np.all(np.abs(g["x"] - r["x"]) <= 1e-6, axis=1)
    assert same.mean() >= 0.98, f"{(~same).sum()} of {B} branch solutions differ"
    rel = np.abs(g["f"] - r["f"])[same] / np.maximum(1.0, np.abs(r["f"][same]))
    assert rel.max() <= 1e-8


@pytest.mark.parametrize("tr_norm", [0, 1])
def test_trust_region_norm_readings_match_oracle(tr_norm):
    # options.tr_norm 0: the CG iterate of the preconditioned system is bounded,
    # ||L^T w|| <= delta (as Algorithm 1 prints it; the default); 1: ||w||_2 <= delta.  The GPU
    # forms the first from CG recurrences, the oracle from the iterate itself.
    d = synth.dense_batch(160, 32, seed_index=7)
    g = gpu_solve(d, n=32, tr_norm=tr_norm)
    r = oracle_solve(d, tr_norm=tr_norm)
    assert_convex_parity(g, r, d["l"], d["u"])
    same_path = g["iters"] == r["iters"]
    assert same_path.mean() >= 0.95
    # the final radius, on the problems that took the same path
    np.testing.assert_allclose(g["delta"][same_path], r["delta"][same_path], rtol=1e-6)
    br = synth.branch_batch(160, seed_index=9)
    for group in (1, 4):
        g = gpu_solve(br, n=4, group=group, tr_norm=tr_norm)
        r = oracle_solve(br, tr_norm=tr_norm)
        assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
        same = np.all(np.abs(g["x"] - r["x"]) <= 1e-6, axis=1)
        assert same.mean() >= 0.98
        assert np.mean(g["iters"] == r["iters"]) >= 0.95


def test_hessian_norm_cauchy_option_matches_oracle():
    # options.cauchy_norm = 1: the Cauchy trial's trust-region test in the model
    # Hessian's norm (s'Hs)^(1/2) where s'Hs > 0, against the oracle with the same option
    d = synth.dense_batch(160, 32, seed_index=17)
    g = gpu_solve(d, n=32, cauchy_norm=1)
    r = oracle_solve(d, cauchy_norm=1)
    assert_convex_parity(g, r, d["l"], d["u"])
    assert np.mean(g["iters"] == r["iters"]) >= 0.95
    br = synth.branch_batch(160, seed_index=19)
    for group in (1, 4):
        g = gpu_solve(br, n=4, group=group, cauchy_norm=1)
        r = oracle_solve(br, cauchy_norm=1)
        assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
        same = np.all(np.abs(g["x"] - r["x"]) <= 1e-6, axis=1)
        assert same.mean() >= 0.98
        assert np.mean(g["iters"] == r["iters"]) >= 0.95
    gr = synth.genramp_batch(96, 24, seed_index=21)
    g = gpu_solve(gr, n=24, cauchy_norm=1)
    r = oracle_solve(gr, cauchy_norm=1)
    assert np.all(g["status"] == native.TRON_CONVERGED) and np.all(r["status"] == 0)
    np.testing.assert_allclose(g["x"], r["x"], rtol=0, atol=1e-6)


def test_branch_default_group_follows_batch_size():
    # the library's mapping of the branch problems: four lanes per problem up to 96
    # problems per SM sub-partition, two lanes beyond; an explicit group wins
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    lim = 96 * 4 * nsm
    for B, want in ((256, 4), (lim, 4), (lim + 1, 2)):
        tb = TronBatch(native.TRON_OBJ_ACOPF_BRANCH, B, n=4)
        assert tb.choices()[0]["group"] == want, (B, tb.choices())
        tb.close()
    tb = TronBatch(native.TRON_OBJ_ACOPF_BRANCH, 256, n=4, opts=options(group=1))
    assert tb.choices()[0]["group"] == 1
    tb.close()


def test_branch_groups_agree_with_line_limits_active():
    # tight line limits so the penalty of eq. exp-branch is active on many branches: the
    # four-lane evaluator (reduce-scatter of the Gauss-Newton terms), the two-lane one
    # (each lane its own direction's limit) and the one-lane one reach the same points,
    # and all are KKT points by the oracle's gradient
    d = synth.branch_batch(200, seed_index=83)
    d["params"] = d["params"].copy()
    d["params"][:, 32] *= 0.05
    a = gpu_solve(d, n=4, group=1)
    b = gpu_solve(d, n=4, group=4)
    c = gpu_solve(d, n=4, group=2)
    r = oracle_solve(d)
    for g in (a, b, c):
        assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
        for p in range(200):
            assert _branch_kkt(d["params"][p], g["x"][p], d["l"][p], d["u"][p]) <= 1e-6 * 1.01
    for g in (a, c):
        same = np.all(np.abs(g["x"] - b["x"]) <= 1e-6, axis=1)
        assert same.mean() >= 0.98
    same_r = np.all(np.abs(b["x"] - r["x"]) <= 1e-6, axis=1)
    assert same_r.mean() >= 0.98


def test_hs45_gpu_matches_printed_solution():
    for n in range(2, 9):
        d = synth.hs45_batch(33, n)
        g = gpu_solve(d, n=n)
        assert np.all(g["status"] == native.TRON_CONVERGED)
        np.testing.assert_allclose(g["x"], np.tile(np.arange(1, n + 1), (33, 1)), atol=1e-9)


def test_uneven_sizes_one_batch():
    d = synth.uneven_batch(400, seed_index=3, sizes=(4, 6, 8, 16, 32),
                           probs=(0.4, 0.2, 0.15, 0.15, 0.1))
    nv = d["nvec"]
    g = gpu_solve(d, n_list=nv)
    r = oracle_solve(d, n_list=nv)
    classes = {min(c for c in (4, 8, 16, 32) if n <= c) for n in nv.tolist()}
    assert g["launches"] == len(classes)   # one launch per size class
    assert np.all(g["status"] == 0) and np.all(r["status"] == 0)
    np.testing.assert_allclose(g["x"], r["x"], rtol=0, atol=1e-6)


def test_uneven_full_size_range_persistent_and_autotuned():
    d = synth.uneven_batch(900, seed_index=3)      # n in {4, 6, 8, 16, 32, 64, 128}
    nv = d["nvec"]
    plain = gpu_solve(d, n_list=nv)
    pers = gpu_solve(d, n_list=nv, schedule=native.TRON_SCHED_PERSISTENT)
    for k in ("x", "f", "pg", "iters", "status", "delta"):
        np.testing.assert_array_equal(plain[k], pers[k])
    assert pers["launches"] == len({min(c for c in (4, 8, 16, 32, 64, 128) if n <= c)
                                    for n in nv.tolist()})
    r = oracle_solve(d, n_list=nv)
    assert np.all(plain["status"] == 0) and np.all(r["status"] == 0)
    np.testing.assert_allclose(plain["x"], r["x"], rtol=0, atol=1e-6)
    # autotuned variants: same solutions within the tolerance
    tb = TronBatch(2, nv.size, n_list=nv, opts=options(schedule=native.TRON_SCHED_PERSISTENT))
    P, L, U, X0, D0 = (_t(d["params"]), _t(d["l"]), _t(d["u"]), _t(d["x0"]), _t(d["delta0"]))
    ch = tb.autotune(P, L, U, X0, D0, sample=256)
    assert [c["N"] for c in ch] == sorted({c["N"] for c in ch}, reverse=True)
    assert all(c["warps_per_block"] in (1, 2, 3, 4, 5, 6, 7, 8) for c in ch)
    np.testing.assert_array_equal(X0.cpu().numpy(), d["x0"])   # inputs untouched
    x, de = X0.clone(), D0.clone()
    out = tb.solve(P, L, U, x, de)
    torch.cuda.synchronize()
    assert np.all(out["status"].cpu().numpy() == 0)
    np.testing.assert_allclose(x.cpu().numpy(), r["x"], rtol=0, atol=1e-6)
    tb.close()


def _same_up_to_contraction(a, b):
    # the plain and persistent kernels run the same solver code, compiled into two
    # kernels whose fused multiply-adds may differ in the last bit
    np.testing.assert_array_equal(a["status"], b["status"])
    np.testing.assert_allclose(a["x"], b["x"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(a["f"], b["f"], rtol=1e-12, atol=0)
    assert np.mean(a["iters"] == b["iters"]) >= 0.98


def test_persistent_equals_plain():
    d = synth.dense_batch(500, 32, seed_index=7)
    a = gpu_solve(d, n=32)
    b = gpu_solve(d, n=32, schedule=native.TRON_SCHED_PERSISTENT)
    _same_up_to_contraction(a, b)
    d = synth.branch_batch(300, seed_index=8)
    for grp in (1, 4):
        a = gpu_solve(d, n=4, group=grp)
        b = gpu_solve(d, n=4, group=grp, schedule=native.TRON_SCHED_PERSISTENT)
        _same_up_to_contraction(a, b)


@pytest.mark.parametrize("mixed", [False, True])
def test_concurrent_solves_on_two_streams_equal_sequential(mixed):
    # one handle, four solves of different batches alternating between two streams (each
    # takes its own work counters): the same bits as solving them one after another
    if mixed:
        # one size layout, four starting points inside the box
        base = synth.uneven_batch(600, seed_index=90)
        ds = [dict(base, x0=base["x0"] + 0.01 * i) for i in range(4)]
        kw = dict(n=None, n_list=base["nvec"])
    else:
        ds = [synth.dense_batch(800, 32, seed_index=95 + i) for i in range(4)]
        kw = dict(n=32, n_list=None)
    refs = [gpu_solve(d, schedule=native.TRON_SCHED_PERSISTENT, **kw) for d in ds]
    B = ds[0]["delta0"].shape[0]
    tb = TronBatch(2, B, n=kw["n"], n_list=kw["n_list"],
                   opts=options(schedule=native.TRON_SCHED_PERSISTENT))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for i, d in enumerate(ds):
        st = streams[i % 2]
        with torch.cuda.stream(st):
            x, dl = _t(d["x0"]), _t(d["delta0"])
            outs.append(tb.solve(_t(d["params"]), _t(d["l"]), _t(d["u"]), x, dl, stream=st))
    torch.cuda.synchronize()
    tb.close()
    for o, r in zip(outs, refs):
        for k in ("x", "delta", "f", "pg", "iters", "status"):
            np.testing.assert_array_equal(o[k].cpu().numpy(), r[k], err_msg=k)


def test_ctas_per_sm_changes_the_schedule_not_the_results():
    d = synth.dense_batch(900, 32, seed_index=97)
    a = gpu_solve(d, n=32, schedule=native.TRON_SCHED_PERSISTENT)
    b = gpu_solve(d, n=32, schedule=native.TRON_SCHED_PERSISTENT, ctas_per_sm=2)
    for k in ("x", "f", "pg", "iters", "status", "delta"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    with pytest.raises(native.TronError, match="EINVAL"):
        TronBatch(2, 4, n=8, opts=options(ctas_per_sm=-1))


def _host(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).pin_memory()


@pytest.mark.parametrize("case", ["dense32", "mixed", "hs45"])
def test_host_buffer_path_equals_device_path(case):
    # three calls in flight through tron_batch_solve_host (shared inputs, distinct
    # outputs, the two device buffer sets reused) give the device path's bits
    if case == "dense32":
        d, n, n_list = synth.dense_batch(700, 32, seed_index=12), 32, None
    elif case == "mixed":
        d = synth.uneven_batch(900, seed_index=13)
        n, n_list = None, d["nvec"]
    else:
        d, n, n_list = synth.hs45_batch(50, 6), 6, None
    ref = gpu_solve(d, n=n, n_list=n_list, schedule=native.TRON_SCHED_PERSISTENT)
    B = d["delta0"].shape[0]
    tb = TronBatch(d["kind"], B, n=n if n_list is None else None, n_list=n_list,
                   opts=options(schedule=native.TRON_SCHED_PERSISTENT))
    tb.host_enable()
    params = _host(d["params"]) if np.size(d["params"]) else None
    ins = [params, _host(d["l"]), _host(d["u"]), _host(d["x0"]), _host(d["delta0"])]
    outs = [tb.host_outputs(int(np.size(d["x0"]))) for _ in range(3)]
    for o in outs:
        tb.solve_host(*ins, o)
    tb.host_sync()
    tb.close()
    for o in outs:
        for k in ("x", "delta", "f", "pg", "iters", "status"):
            np.testing.assert_array_equal(o[k].numpy().reshape(ref[k].shape), ref[k],
                                          err_msg=k)


def test_host_buffer_path_requires_enable():
    d = synth.dense_batch(4, 8, seed_index=14)
    tb = TronBatch(2, 4, n=8)
    with pytest.raises(native.TronError, match="EINVAL"):
        tb.solve_host(_host(d["params"]), _host(d["l"]), _host(d["u"]), _host(d["x0"]),
                      _host(d["delta0"]), tb.host_outputs(32))
    tb.close()


def test_edge_cases_status_codes():
    n = 6
    d = synth.dense_batch(8, n, seed_index=9)
    d["l"][1, 2] = d["u"][1, 2] + 1.0                     # l > u
    d["params"][2, n * n] = np.nan                        # non-finite record
    d["x0"][3] = 50.0                                     # x0 outside the box
    d["delta0"][4] = -1.0                                 # automatic initial radius
    g = gpu_solve(d, n=n)
    r = oracle_solve(d)
    np.testing.assert_array_equal(g["status"], r["status"])
    assert g["status"][1] == native.TRON_BAD_BOUNDS and g["iters"][1] == 0
    np.testing.assert_array_equal(g["x"][1], d["x0"][1])   # left as given
    assert g["status"][2] == native.TRON_NONFINITE
    for p in (0, 3, 4, 5, 6, 7):
        assert g["status"][p] == 0
        np.testing.assert_allclose(g["x"][p], r["x"][p], atol=1e-6)
    # iteration cap
    g = gpu_solve(d, n=n, max_outer=1, gtol=1e-300)
    assert np.all(g["status"][[0, 3, 4]] == native.TRON_MAX_ITER)
    assert np.all(g["iters"][[0, 3, 4]] == 1)


@pytest.mark.parametrize("group", [1, 2, 4])
def test_branch_edge_cases_status_codes(group):
    # the branch evaluator on one and four lanes: l > u, a non-finite record, x0 outside
    # the box, an automatic initial radius; status codes as the oracle's, converged
    # results KKT points by the oracle's gradient
    d = synth.branch_batch(12, seed_index=84)
    d = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in d.items()}
    d["l"][1, 2] = d["u"][1, 2] + 1.0
    d["params"][2, 5] = np.nan
    d["params"][5, 20] = np.inf                  # a target: f is infinite everywhere
    d["params"][6, 32] = np.inf                  # no line limit: the penalty never applies
    d["params"][7, 32] = np.nan                  # m > 0 is false for NaN, as in the oracle
    d["params"][8, 33] = np.inf                  # line weight, unused while no line is over
    d["x0"][3] = [1.5, 0.2, 20.0, -20.0]
    d["delta0"][4] = -1.0
    g = gpu_solve(d, n=4, group=group)
    r = oracle_solve(d)
    np.testing.assert_array_equal(g["status"], r["status"])
    assert g["status"][1] == native.TRON_BAD_BOUNDS and g["iters"][1] == 0
    np.testing.assert_array_equal(g["x"][1], d["x0"][1])
    assert g["status"][2] == native.TRON_NONFINITE
    assert g["status"][5] == native.TRON_NONFINITE
    for p in (0, 3, 4, 6, 7, 8, 9, 10, 11):
        assert g["status"][p] == native.TRON_CONVERGED
        assert np.all(g["x"][p] >= d["l"][p]) and np.all(g["x"][p] <= d["u"][p])
        assert _branch_kkt(d["params"][p], g["x"][p], d["l"][p], d["u"][p]) <= 1e-6 * 1.01


@pytest.mark.parametrize("n", [6, 32, 64])
def test_degenerate_boxes_fixed_variables(n):
    # l = u on some variables (fixed), every variable fixed in one problem, a
    # zero-width box at the unconstrained minimiser's side, and x0 already optimal
    d = synth.dense_batch(12, n, seed_index=70 + n)
    rng = np.random.default_rng(70 + n)
    for p in range(12):
        fix = rng.random(n) < 0.3
        d["l"][p, fix] = d["u"][p, fix] = rng.uniform(-0.5, 0.5, fix.sum())
    d["l"][3] = d["u"][3] = 0.25                                  # everything fixed
    r0 = oracle_solve(d)
    d["x0"][5] = r0["x"][5]                                       # start at the solution
    g = gpu_solve(d, n=n)
    r = oracle_solve(d)
    assert_convex_parity(g, r, d["l"], d["u"])
    fixed = d["l"] == d["u"]
    np.testing.assert_array_equal(g["x"][fixed], d["l"][fixed])
    assert g["iters"][3] == r["iters"][3]
    assert g["iters"][5] <= 1


def test_empty_batch_is_noop():
    tb = TronBatch(native.TRON_OBJ_DENSE_QUARTIC, 0, n=8)
    e = torch.empty(0, dtype=torch.float64, device=DEV)
    out = tb.solve(e, e, e, e, e)
    assert tb.last_launches == 0
    tb.close()


def test_full_size_dense_workload_sampled():
    """10,000 problems, n = 32, in the benchmark's launch configuration; 200 sampled
    problems re-solved by the oracle one by one; all problems satisfy the invariants."""
    d = synth.dense_batch(10000, 32, seed_index=1)
    g = gpu_solve(d, n=32)
    assert np.all(g["status"] == 0)
    assert np.all(g["pg"] <= 1e-6)
    assert np.all(g["x"] >= d["l"]) and np.all(g["x"] <= d["u"])
    idx = np.random.default_rng(0).choice(10000, 200, replace=False)
    sub = {k: (v[idx] if isinstance(v, np.ndarray) and v.ndim and v.shape[0] == 10000 else v)
           for k, v in d.items()}
    r = oracle_solve(sub)
    np.testing.assert_allclose(g["x"][idx], r["x"], rtol=0, atol=1e-6)
    rel = np.abs(g["f"][idx] - r["f"]) / np.maximum(1.0, np.abs(r["f"]))
    assert rel.max() <= 1e-8


def test_full_size_dense_high_active_fraction_in_the_bench_configuration():
    """10,000 problems, n = 32, with c ~ N(0, 16^2) so that about 30 % of the bounds are
    active at the solution (the share the workload description expects; the benchmark's
    c ~ N(0, 4^2) gives 10 %): more Cauchy breakpoints, newly active variables and
    multi-pass subspace loops.  Solved as the benchmark solves (persistent schedule after
    autotuning); 1,000 sampled problems re-solved by the oracle."""
    d = synth.dense_batch(10000, 32, seed_index=41, c_sd=16.0)
    tb = TronBatch(2, 10000, n=32, opts=options(schedule=native.TRON_SCHED_PERSISTENT))
    P, L, U = _t(d["params"]), _t(d["l"]), _t(d["u"])
    tb.autotune(P, L, U, _t(d["x0"]), _t(d["delta0"]), sample=4096)
    x, delta = _t(d["x0"]), _t(d["delta0"])
    out = tb.solve(P, L, U, x, delta)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    tb.close()
    assert np.all(g["status"] == 0)
    assert np.all(g["pg"] <= 1e-6)
    active = np.mean((g["x"] <= d["l"]) | (g["x"] >= d["u"]))
    assert 0.25 <= active <= 0.4, active
    idx = np.random.default_rng(1).choice(10000, 1000, replace=False)
    sub = {k: (v[idx] if isinstance(v, np.ndarray) and v.ndim and v.shape[0] == 10000 else v)
           for k, v in d.items()}
    r = oracle_solve(sub)
    assert np.all(r["status"] == oracle.CONVERGED)
    np.testing.assert_allclose(g["x"][idx], r["x"], rtol=0, atol=1e-6)
    rel = np.abs(g["f"][idx] - r["f"]) / np.maximum(1.0, np.abs(r["f"]))
    assert rel.max() <= 1e-8
    # the same active set on the sampled problems
    act_g = (g["x"][idx] <= d["l"][idx]) | (g["x"][idx] >= d["u"][idx])
    act_o = (r["x"] <= d["l"][idx]) | (r["x"] >= d["u"][idx])
    assert np.mean(act_g == act_o) >= 0.999


def test_pivot_reciprocal_against_ieee_division():
    # the factorization's 1/d: hardware estimate + one Newton step (division from
    # 2^1022 up); relative error against the correctly rounded 1/d <= 2^-38 over the
    # positive normal range, powers of two and their neighbours included
    rng = np.random.default_rng(5)
    e = rng.uniform(-1022.0, 1023.99, 1 << 20)
    a = np.ldexp(1.0, 0) * np.exp2(e)
    p2 = np.ldexp(1.0, np.arange(-1022, 1024))
    a = np.concatenate([a, p2, np.nextafter(p2, 0.0), np.nextafter(p2, np.inf),
                        [np.finfo(float).tiny, np.finfo(float).max, 1.0, 3.0, 1e-300, 1e300]])
    a = a[np.isfinite(a) & (a >= np.finfo(float).tiny)]
    d_a = _t(a)
    d_out = torch.empty_like(d_a)
    lib = native.load()
    assert lib.tron_test_pivot_rcp(d_a.data_ptr(), d_out.data_ptr(), a.size,
                                   torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    got = d_out.cpu().numpy()
    ref = 1.0 / a
    rel = np.abs(got - ref) / ref
    assert np.all(np.isfinite(got))
    assert rel.max() <= 2.0 ** -38, (rel.max(), a[np.argmax(rel)])
    # from 2^1022 up the hook divides: exact
    big = a >= 2.0 ** 1022
    np.testing.assert_array_equal(got[big], ref[big])


def _arith(op, a, b=None):
    lib = native.load()
    d_a = _t(a)
    d_b = _t(b) if b is not None else None
    d_out = torch.empty_like(d_a)
    assert lib.tron_test_arith(op, d_a.data_ptr(), d_b.data_ptr() if d_b is not None else None,
                               d_out.data_ptr(), a.size,
                               torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


def _within_one_ulp(got, ref):
    # got is one of the two doubles around the exact value when it is within one ulp of
    # the correctly rounded ref (the spacing at |ref|, the larger one at a power of two)
    with np.errstate(over="ignore"):
        return np.abs(got - ref) <= np.spacing(np.abs(ref))


def test_solver_quotient_against_ieee_division():
    # the CG step lengths, trqsol's root and the radius update divide with the refined
    # hardware reciprocal: faithful everywhere, correctly rounded but for rare midpoint
    # cases, and exactly IEEE (signed zeros, infinities, NaN, subnormals) outside its range
    rng = np.random.default_rng(11)
    n = 1 << 20
    a = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-1000, 1000, n)) * rng.choice([-1.0, 1.0], n)
    b = np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-1000, 1000, n)) * rng.choice([-1.0, 1.0], n)
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -5e-324, np.finfo(float).tiny,
                   np.finfo(float).max, 1.0, -1.0, 3.0, 2.0 ** 1022, 2.0 ** -1021, 1e-300, 1e300])
    sa, sb = np.meshgrid(sp, sp)
    a = np.concatenate([a, sa.ravel(), np.ldexp(1.0, np.arange(-1000, 1000)), rng.normal(size=4096)])
    b = np.concatenate([b, sb.ravel(), np.full(2000, 3.0), rng.normal(size=4096)])
    with np.errstate(all="ignore"):
        ref = a / b
    got = _arith(1, a, b)
    fin = np.isfinite(ref) & (ref != 0.0)
    assert np.all(_within_one_ulp(got[fin], ref[fin])), a[fin][~_within_one_ulp(got[fin], ref[fin])][:4]
    assert np.mean(got[fin] != ref[fin]) <= 1e-3
    # NaN where IEEE gives NaN; zeros and infinities with their signs
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    rest = ~fin & ~np.isnan(ref)
    np.testing.assert_array_equal(got[rest].view(np.int64), ref[rest].view(np.int64))


def test_solver_square_root_against_ieee_sqrt():
    rng = np.random.default_rng(12)
    n = 1 << 20
    x = np.ldexp(rng.uniform(1.0, 4.0, n), 2 * rng.integers(-511, 511, n))
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -1.0, 5e-324, np.finfo(float).tiny,
                   np.finfo(float).max, 1.0, 2.0, 4.0, 0.25, 1e-300, 1e300])
    sq = rng.uniform(0.5, 2.0, 4096)
    x = np.concatenate([x, sp, np.ldexp(1.0, np.arange(-1074, 1024)), sq * sq])
    with np.errstate(all="ignore"):
        ref = np.sqrt(x)
    got = _arith(2, x)
    fin = np.isfinite(ref) & (ref > 0.0)
    assert np.all(_within_one_ulp(got[fin], ref[fin])), x[fin][~_within_one_ulp(got[fin], ref[fin])][:4]
    assert np.mean(got[fin] != ref[fin]) <= 1e-3
    np.testing.assert_array_equal(np.isnan(got), np.isnan(ref))
    rest = ~fin & ~np.isnan(ref)
    np.testing.assert_array_equal(got[rest].view(np.int64), ref[rest].view(np.int64))
    # exact squares: powers of two have exact roots, which a faithful result must hit
    p2 = np.ldexp(1.0, 2 * np.arange(-500, 500))
    np.testing.assert_array_equal(_arith(2, p2), np.ldexp(1.0, np.arange(-500, 500)))


@pytest.mark.parametrize("group", [1, 4])
@pytest.mark.parametrize("sched", ["plain", "persistent"])
def test_small_batch_spread_over_warps_gives_the_same_bits(group, sched):
    # 256 problems alone: fewer problems per warp (one per warp here), so that each SM
    # sub-partition holds one warp; the same 256 inside a batch of 8,192 are packed as
    # many per warp as fit.  A problem's arithmetic does not depend on its place.
    big = synth.branch_batch(8192, seed_index=41)
    keys = ("params", "l", "u", "x0", "delta0")
    small = {k: big[k][:256] for k in keys}
    small["kind"] = big["kind"]
    s = native.TRON_SCHED_PLAIN if sched == "plain" else native.TRON_SCHED_PERSISTENT
    g_small = gpu_solve(small, n=4, group=group, schedule=s)
    g_big = gpu_solve(big, n=4, group=group, schedule=s)
    for k in ("x", "f", "pg", "delta", "iters", "status"):
        np.testing.assert_array_equal(g_small[k], g_big[k][:256], err_msg=k)
    assert np.all(g_small["status"] == native.TRON_CONVERGED)


def test_branch_sine_and_cosine_against_the_library():
    # the branch objective's sin and cos of theta_i - theta_j: a Taylor series for
    # |x| <= pi/4, the library's functions outside; within one ulp of the correctly
    # rounded value everywhere (numpy's as the reference), signed zero kept
    rng = np.random.default_rng(13)
    q = np.pi / 4
    x = np.concatenate([rng.uniform(-q, q, 1 << 20), rng.uniform(-4 * np.pi, 4 * np.pi, 1 << 16),
                        np.ldexp(1.0, -np.arange(1, 1000)), -np.ldexp(1.0, -np.arange(1, 1000)),
                        [0.0, -0.0, q, -q, np.nextafter(q, 1.0), np.nextafter(q, 0.0), 1e5]])
    for op, fn in ((3, np.sin), (4, np.cos)):
        got = _arith(op, x)
        ref = fn(x)
        ok = np.abs(got - ref) <= np.spacing(np.abs(ref))
        assert np.all(ok), (op, x[~ok][:4], got[~ok][:4], ref[~ok][:4])
        inside = np.abs(x) <= q
        assert np.mean(got[inside] != ref[inside]) <= 0.05
    s0 = _arith(3, np.array([0.0, -0.0]))
    assert s0[0] == 0.0 and s0[1] == 0.0 and np.signbit(s0[1]) and not np.signbit(s0[0])
    np.testing.assert_array_equal(_arith(4, np.array([0.0, -0.0])), [1.0, 1.0])


def test_full_size_uneven_workload_sampled():
    # the bench's uneven workload (100,000 problems, n in {4, 6, 8, 16, 32, 64, 128}) in
    # the bench's launch configuration: persistent schedule, autotuned variants, every
    # size class at once; the oracle solves a stratified sample, 40 problems per class
    d = synth.uneven_batch(100000, seed_index=3)
    nv = d["nvec"]
    tb = TronBatch(2, nv.size, n_list=nv, opts=options(schedule=native.TRON_SCHED_PERSISTENT))
    P, L, U, X0, D0 = (_t(d["params"]), _t(d["l"]), _t(d["u"]), _t(d["x0"]), _t(d["delta0"]))
    tb.autotune(P, L, U, X0, D0, sample=8192)
    x, de = X0.clone(), D0.clone()
    out = tb.solve(P, L, U, x, de)
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    xs = x.cpu().numpy()
    tb.close()
    assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
    assert np.all(g["pg"] <= 1e-6)
    voff = np.concatenate([[0], np.cumsum(nv)])
    poff = np.concatenate([[0], np.cumsum(nv * nv + 2 * nv)])
    cls = np.array([min(c for c in (4, 8, 16, 32, 64, 128) if n <= c) for n in nv.tolist()])
    rng = np.random.default_rng(2)
    idx = np.sort(np.concatenate([
        rng.choice(np.flatnonzero(cls == c), min(40, int((cls == c).sum())), replace=False)
        for c in np.unique(cls)]))
    vec = lambda a: np.concatenate([a[voff[i]:voff[i + 1]] for i in idx])
    sub = dict(kind=2, nvec=nv[idx], l=vec(d["l"]), u=vec(d["u"]), x0=vec(d["x0"]),
               delta0=d["delta0"][idx],
               params=np.concatenate([d["params"][poff[i]:poff[i + 1]] for i in idx]))
    r = oracle_solve(sub, n_list=sub["nvec"])
    assert np.all(r["status"] == oracle.CONVERGED)
    np.testing.assert_allclose(vec(xs), r["x"], rtol=0, atol=1e-6)
    rel = np.abs(g["f"][idx] - r["f"]) / np.maximum(1.0, np.abs(r["f"]))
    assert rel.max() <= 1e-8, rel.max()


@pytest.mark.parametrize("n,B", [(16, 300), (32, 300), (128, 40)])
def test_dense_indefinite_shifted_factorization_and_negative_curvature(n, B):
    # indefinite Q (a quarter of the eigenvalues in -[0.5, 50]): the factorization needs
    # shifts and the PCG exits on negative curvature (the oracle's counters show both);
    # several local minima can be correct, so every GPU result must be a KKT point by
    # the oracle's own gradient, and where GPU and oracle took the same path (the same
    # iteration count) they must agree as on convex problems
    d = synth.dense_batch(B, n, seed_index=60 + n, neg_frac=0.25)
    g = gpu_solve(d, n=n)
    r = oracle_solve(d)
    c = r["counters"]
    assert c["chol_calls"] > c["subspace_passes"], c   # shift retries happened
    assert c["cg_iters"] > 0, c
    assert np.all(g["status"] == native.TRON_CONVERGED), np.bincount(g["status"])
    assert np.all(r["status"] == oracle.CONVERGED)
    assert np.all(g["x"] >= d["l"]) and np.all(g["x"] <= d["u"])
    for p in range(B):
        _, gr, _ = oracle.eval_obj(oracle.OBJ_DENSE, d["params"][p], g["x"][p])
        assert oracle.pgnorm(g["x"][p], gr, d["l"][p], d["u"][p]) <= 1e-6 * 1.01
    same = g["iters"] == r["iters"]
    assert same.mean() >= 0.8, same.mean()
    np.testing.assert_allclose(g["x"][same], r["x"][same], rtol=0, atol=1e-6)
    rel = np.abs(g["f"][same] - r["f"][same]) / np.maximum(1.0, np.abs(r["f"][same]))
    assert rel.max() <= 1e-8


def test_operation_costs_behind_the_design():
    # the measured facts the solver is built on: a dependent FP64 instruction costs the
    # same with 1 or 32 active lanes; FP64 compare-and-select costs more than an FP64 FMA
    # and far more than the int64 one the solver uses instead; the solver's quotient,
    # square root and sine series are shorter chains than the library's operations
    from paper_2106_14995_gb300.tron import op_latency
    c = {k: op_latency(k, 32) for k in range(13)}
    one = op_latency(0, 1)
    assert abs(one - c[0]) <= 0.1 * c[0], (one, c[0])
    assert c[3] > c[0] and c[4] < 0.5 * c[3], c
    assert c[5] < c[6] and c[7] < c[8] and c[10] < c[9], c
