"""The entry point that allocates no device memory (tron_solve_mixed_noalloc).

It exists for callers that must not allocate device memory from a library call: hosts
whose device memory all belongs to their own pool allocator, where a cudaMalloc beside
the pool fails or fragments it, and processes held to a fixed device-memory budget.
Here it is called through the C ABI twice in a row on two different mixed-size batches
that between them cover every size class (4 to 128), and each result is compared with
the regular handle-based entry point (tron_batch_create + tron_batch_solve) on the same
inputs, and the first batch also with the CPU oracle, within the tolerances of the other
GPU tests.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2106_14995_gb300 import native, synth
from paper_2106_14995_gb300.tron import TronBatch, options

pytestmark = pytest.mark.gpu


def _t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def _outputs(B):
    return dict(f=torch.empty(B, dtype=torch.float64, device="cuda:0"),
                pg=torch.empty(B, dtype=torch.float64, device="cuda:0"),
                iters=torch.empty(B, dtype=torch.int32, device="cuda:0"),
                status=torch.empty(B, dtype=torch.int32, device="cuda:0"))


def _via_handle(d):
    B = d["nvec"].size
    tb = TronBatch(2, B, n_list=d["nvec"], opts=options(schedule=native.TRON_SCHED_PERSISTENT))
    x, delta = _t(d["x0"]), _t(d["delta0"])
    out = tb.solve(_t(d["params"]), _t(d["l"]), _t(d["u"]), x, delta)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    tb.close()
    return res


def _via_noalloc(lib, d, stream):
    B = d["nvec"].size
    n_arr = (C.c_int32 * B)(*d["nvec"].tolist())
    opts = native.tron_options_default()
    P, L, U = _t(d["params"]), _t(d["l"]), _t(d["u"])
    x, delta = _t(d["x0"]), _t(d["delta0"])
    out = _outputs(B)
    torch.cuda.synchronize()
    rc = lib.tron_solve_mixed_noalloc(
        2, B, C.cast(n_arr, C.c_void_p), C.byref(opts), P.data_ptr(), L.data_ptr(),
        U.data_ptr(), x.data_ptr(), delta.data_ptr(), out["f"].data_ptr(),
        out["pg"].data_ptr(), out["iters"].data_ptr(), out["status"].data_ptr(),
        stream.cuda_stream)
    assert rc == 0, lib.tron_last_error()
    stream.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["x"] = x.cpu().numpy()
    res["delta"] = delta.cpu().numpy()
    return res


def test_noalloc_matches_handle_path_on_two_calls_in_a_row():
    import oracle
    lib = native.load()
    stream = torch.cuda.Stream()
    sizes = (4, 6, 8, 16, 32, 64, 128)
    probs = (0.3, 0.2, 0.15, 0.15, 0.1, 0.06, 0.04)
    batches = [synth.uneven_batch(300, seed_index=11, sizes=sizes, probs=probs),
               synth.uneven_batch(450, seed_index=12, sizes=sizes, probs=probs)]
    for k, d in enumerate(batches):  # two calls in a row; the second reuses the scratch
        assert set(np.unique(d["nvec"])) == set(sizes)  # every size class is present
        a = _via_noalloc(lib, d, stream)
        b = _via_handle(d)
        np.testing.assert_array_equal(a["status"], b["status"])
        assert np.all(a["status"] == native.TRON_CONVERGED)
        assert np.all(a["pg"] <= 1e-6)
        np.testing.assert_allclose(a["x"], b["x"], rtol=0, atol=1e-6)
        rel = np.abs(a["f"] - b["f"]) / np.maximum(1.0, np.abs(b["f"]))
        assert rel.max() <= 1e-8
        if k == 0:  # and against the CPU oracle
            r = oracle.tron_batch(2, d["params"], d["l"], d["u"], d["x0"], d["delta0"],
                                  n=d["nvec"], nthreads=8)
            assert np.all(r["status"] == oracle.CONVERGED)
            np.testing.assert_allclose(a["x"], r["x"], rtol=0, atol=1e-6)
            rel = np.abs(a["f"] - r["f"]) / np.maximum(1.0, np.abs(r["f"]))
            assert rel.max() <= 1e-8


def test_noalloc_rejects_batches_beyond_its_capacity():
    lib = native.load()
    too_many = (1 << 18) + 1
    rc = lib.tron_solve_mixed_noalloc(2, too_many, None, None, None, None, None, None, None,
                                      None, None, None, None, None)
    assert rc == 1  # TRON_EINVAL
    assert b"capacity" in lib.tron_last_error()
