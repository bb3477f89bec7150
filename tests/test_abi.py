"""C-ABI library: builds, loads without a GPU, exports every declared symbol; option
defaults agree with the oracle's readings; argument errors are reported, not thrown."""
import ctypes as C
import os
import re

import pytest

from paper_2106_14995_gb300 import _build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return C.CDLL(_build.LIB)


def test_library_exports_every_declared_symbol(lib):
    decl = _declared_functions()
    assert "tron_batch_solve" in decl and "tron_batch_create" in decl
    for name in decl:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_options_defaults_match_oracle_readings():
    import oracle
    o = native.tron_options_default()
    r = oracle.default_opts()
    for f in ("gtol", "max_outer", "max_trials", "mu0", "mu1", "interpf", "extrapf",
              "proj_shrink", "eta0", "eta1", "eta2", "sigma1", "sigma3", "delta_max",
              "delta_min_rel", "cg_rtol", "shift_frac", "max_shift", "ared_guard", "tr_norm",
              "cauchy_norm"):
        assert getattr(o, f) == getattr(r, f), f
    assert o.group == 0 and o.schedule == native.TRON_SCHED_PLAIN
    assert o.split_outer == 0 and list(o.reserved) == [0, 0]


def test_status_numbering_matches_oracle():
    import oracle
    assert native.TRON_CONVERGED == oracle.CONVERGED
    assert native.TRON_MAX_ITER == oracle.MAX_ITER
    assert native.TRON_TR_TOO_SMALL == oracle.TR_TOO_SMALL
    assert native.TRON_CHOL_FAIL == oracle.CHOL_FAIL
    assert native.TRON_NONFINITE == oracle.NONFINITE
    assert native.TRON_BAD_BOUNDS == oracle.BAD_BOUNDS


def test_argument_errors_are_codes(lib):
    L = native.load()
    h = C.c_void_p()
    # bad kind is rejected before any CUDA call
    rc = L.tron_batch_create(C.byref(h), 99, 10, None, 4, None, None)
    assert rc == 1
    assert b"kind" in L.tron_last_error()
    rc = L.tron_batch_create(None, 1, 10, None, 4, None, None)
    assert rc == 1
    o = native.tron_options_default()
    o.group = 3
    rc = L.tron_batch_create(C.byref(h), 2, 10, None, 32, C.byref(o), None)
    assert rc == 1
    assert L.tron_options_default(None) == 1
    # the ADMM branch launch takes one, two or four lanes per branch problem
    o.group = 3
    rc = L.admm_pool_create(C.byref(h), 10, 10, 10, 1, 16, C.byref(o), None)
    assert rc == 1
    assert b"group" in L.tron_last_error()
    assert L.tron_batch_solve(None, None, None, None, None, None, None, None, None, None,
                              None) == 1
    L.tron_batch_destroy(None)  # ignored
