"""ctypes binding of the C ABI (include/tron.h, include/admm.h).

Argument marshalling only: every step of a solve runs in the CUDA kernels of
libexatron_gb300.so.  The functions keep the C names; device buffers are torch CUDA
tensors (their data pointers are passed) and streams are torch CUDA streams.  There is
no fallback: a missing library or a failing call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

TRON_OBJ_ACOPF_BRANCH, TRON_OBJ_DENSE_QUARTIC, TRON_OBJ_HS45, TRON_OBJ_GEN_RAMP = 1, 2, 3, 4
TRON_CONVERGED, TRON_MAX_ITER, TRON_TR_TOO_SMALL, TRON_CHOL_FAIL, TRON_NONFINITE, \
    TRON_BAD_BOUNDS = range(6)
TRON_SCHED_PLAIN, TRON_SCHED_PERSISTENT = 0, 1
ERR_NAMES = {0: "TRON_OK", 1: "TRON_EINVAL", 2: "TRON_ENOMEM", 3: "TRON_ECUDA",
             4: "TRON_EUNSUPPORTED"}


class TronOptions(C.Structure):
    _fields_ = [
        ("gtol", C.c_double), ("max_outer", C.c_int32), ("max_trials", C.c_int32),
        ("mu0", C.c_double), ("mu1", C.c_double), ("interpf", C.c_double),
        ("extrapf", C.c_double), ("proj_shrink", C.c_double), ("eta0", C.c_double),
        ("eta1", C.c_double), ("eta2", C.c_double), ("sigma1", C.c_double),
        ("sigma3", C.c_double), ("delta_max", C.c_double), ("delta_min_rel", C.c_double),
        ("cg_rtol", C.c_double), ("shift_frac", C.c_double), ("max_shift", C.c_int32),
        ("group", C.c_int32), ("ared_guard", C.c_double), ("schedule", C.c_int32),
        ("warps_per_block", C.c_int32), ("layout", C.c_int32), ("cholesky", C.c_int32),
        ("ctas_per_sm", C.c_int32), ("tr_norm", C.c_int32), ("cauchy_norm", C.c_int32),
        ("split_outer", C.c_int32),
        ("reserved", C.c_int32 * 2),
    ]


class AdmmNetwork(C.Structure):
    _fields_ = [
        ("nbus", C.c_int32), ("nbranch", C.c_int32), ("ngen", C.c_int32),
        ("br_from", C.c_void_p), ("br_to", C.c_void_p), ("br_coef", C.c_void_p),
        ("br_smax2", C.c_void_p), ("gen_bus", C.c_void_p), ("gen_c2", C.c_void_p),
        ("gen_c1", C.c_void_p), ("gen_pmin", C.c_void_p), ("gen_pmax", C.c_void_p),
        ("gen_qmin", C.c_void_p), ("gen_qmax", C.c_void_p), ("bus_pd", C.c_void_p),
        ("bus_qd", C.c_void_p), ("bus_gsh", C.c_void_p), ("bus_bsh", C.c_void_p),
        ("rho", C.c_double), ("rho_line", C.c_double), ("vmin", C.c_double),
        ("vmax", C.c_double),
    ]


class AdmmStateView(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in (
        "br_x", "br_delta", "br_lam", "br_val", "br_tilde", "bus_w", "bus_th", "gen_pq",
        "gen_lam", "gen_tilde")] + [("iteration", C.c_int64)]


class TronError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load (building in-tree if needed) libexatron_gb300.so; raises if impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise TronError("libexatron_gb300.so is missing; run __graft_entry__.build()")
        L = C.CDLL(_build.LIB)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "tron_options_default": (I32, [C.POINTER(TronOptions)]),
            "tron_batch_create": (I32, [C.POINTER(P), I32, I64, P, I32,
                                        C.POINTER(TronOptions), P]),
            "tron_batch_set_options": (I32, [P, C.POINTER(TronOptions)]),
            "tron_batch_solve": (I32, [P, P, P, P, P, P, P, P, P, P, P]),
            "tron_batch_last_launches": (I32, [P]),
            "tron_batch_autotune": (I32, [P, P, P, P, P, P, I32, P]),
            "tron_batch_buckets": (I32, [P]),
            "tron_batch_get_choice": (I32, [P, I32, P, P, P, P, P]),
            "tron_solve_mixed_noalloc": (I32, [I32, I64, P, C.POINTER(TronOptions), P, P, P, P,
                                               P, P, P, P, P, P]),
            "tron_batch_host_enable": (I32, [P]),
            "tron_batch_solve_host": (I32, [P, P, P, P, P, P, P, P, P, P, P, P]),
            "tron_batch_host_sync": (I32, [P]),
            "tron_batch_destroy": (None, [P]),
            "tron_last_error": (C.c_char_p, []),
            "tron_version": (C.c_char_p, []),
            "tron_test_pivot_rcp": (I32, [P, P, I64, P]),
            "tron_test_arith": (I32, [I32, P, P, P, I64, P]),
            "tron_bench_fp64_fma": (I32, [P, I32, I32, I64, P]),
            "tron_bench_op_latency": (I32, [I32, I32, P, P]),
            "tron_bench_op_chain": (I32, []),
            "admm_create": (I32, [C.POINTER(P), C.POINTER(AdmmNetwork), C.POINTER(TronOptions),
                                  P]),
            "admm_step": (I32, [P, I32, P, P, P]),
            "admm_residual_history": (I32, [P, I64, I64, P, P, P]),
            "admm_get_state": (I32, [P, C.POINTER(AdmmStateView), P]),
            "admm_set_state": (I32, [P, C.POINTER(AdmmStateView), P]),
            "admm_branch_status_counts": (I32, [P, P, P]),
            "admm_iterations": (I64, [P]),
            "admm_history_capacity": (I64, [P]),
            "admm_launches_per_iteration": (I32, []),
            "admm_pool_launches_per_iteration": (I32, [P]),
            "admm_mp_launches_per_iteration": (I32, [P]),
            "admm_destroy": (None, [P]),
            "admm_pool_create": (I32, [C.POINTER(P), I32, I32, I32, I32, I32,
                                       C.POINTER(TronOptions), P]),
            "admm_pool_add": (I32, [P, C.POINTER(AdmmNetwork), C.POINTER(I32), P]),
            "admm_pool_remove": (I32, [P, I32, P]),
            "admm_pool_step": (I32, [P, I32, P]),
            "admm_pool_residuals": (I32, [P, P, P, P, P]),
            "admm_pool_history": (I32, [P, I32, I64, I64, P, P, P]),
            "admm_pool_get_state": (I32, [P, I32, C.POINTER(AdmmStateView), P]),
            "admm_pool_set_state": (I32, [P, I32, C.POINTER(AdmmStateView), P]),
            "admm_pool_live": (I32, [P]),
            "admm_pool_branch_group": (I32, [P]),
            "admm_pool_destroy": (None, [P]),
            "admm_mp_create": (I32, [C.POINTER(P), C.POINTER(AdmmNetwork), I32, P, P,
                                     C.c_double, C.POINTER(TronOptions), P]),
            "admm_mp_step": (I32, [P, I32, P, P, P]),
            "admm_mp_get_state": (I32, [P, I32, C.POINTER(AdmmStateView), P]),
            "admm_mp_gen_status_counts": (I32, [P, P, P]),
            "admm_mp_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def check(code: int, what: str) -> None:
    if code != 0:
        msg = load().tron_last_error().decode(errors="replace")
        raise TronError(f"{what}: {ERR_NAMES.get(code, code)}: {msg}")


def hptr(t) -> int:
    """Host pointer of a contiguous torch CPU tensor (None -> NULL)."""
    if t is None:
        return 0
    if t.is_cuda:
        raise TronError("expected a host tensor")
    if not t.is_contiguous():
        raise TronError("expected a contiguous tensor")
    return t.data_ptr()


def ptr(t) -> int:
    """Device pointer of a torch tensor (None -> NULL)."""
    if t is None:
        return 0
    if not t.is_cuda:
        raise TronError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise TronError("expected a contiguous tensor")
    return t.data_ptr()


def stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def tron_options_default() -> TronOptions:
    o = TronOptions()
    check(load().tron_options_default(C.byref(o)), "tron_options_default")
    return o


def tron_version() -> str:
    return load().tron_version().decode()
