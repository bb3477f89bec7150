"""CPU FP64 oracle of batched TRON and the component ADMM (arXiv 2106.14995).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` leg of ``bench.py`` are the only callers; the CUDA product path never
imports this package.  The arithmetic lives in ``tron_oracle.c`` (plain C, FP64,
compiled with ``-ffp-contract=off``); this module only marshals numpy arrays.

Functions whose result is pinned by the tests: ``tron_solve``/``tron_batch`` (closed
forms, brute force, the hs45 solution printed in Sec. 4.2, KKT), ``eval_obj`` (finite
differences, autograd, complex power), ``chol_shifted``/``chol`` (numpy), ``trqsol``
(quadratic roots), ``steihaug`` (one iteration when A is positive definite, Sec. 4.3),
``admm_run`` (closed-form bus/generator KKT, residual decay), ``MultiPeriodAdmm`` (equal
to independent single-period runs when no ramp binds; brute force on the generator
chain).
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, "tron_oracle.c")]
_lock = threading.Lock()
_lib = None

OBJ_BRANCH, OBJ_DENSE, OBJ_HS45, OBJ_GENRAMP = 1, 2, 3, 4
CONVERGED, MAX_ITER, TR_TOO_SMALL, CHOL_FAIL, NONFINITE, BAD_BOUNDS = range(6)
STATUS_NAMES = ["CONVERGED", "MAX_ITER", "TR_TOO_SMALL", "CHOL_FAIL", "NONFINITE", "BAD_BOUNDS"]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-O2 -ffp-contract=off)."""
    newest = max(os.path.getmtime(p) for p in _SRC + [os.path.join(_HERE, "oracle.h")])
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= newest):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp] + _SRC + ["-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Opts(C.Structure):
    _fields_ = [
        ("gtol", C.c_double), ("max_outer", C.c_int32), ("max_trials", C.c_int32),
        ("mu0", C.c_double), ("mu1", C.c_double), ("interpf", C.c_double),
        ("extrapf", C.c_double), ("proj_shrink", C.c_double),
        ("eta0", C.c_double), ("eta1", C.c_double), ("eta2", C.c_double),
        ("sigma1", C.c_double), ("sigma3", C.c_double), ("delta_max", C.c_double),
        ("delta_min_rel", C.c_double), ("cg_rtol", C.c_double), ("shift_frac", C.c_double),
        ("max_shift", C.c_int32), ("tr_norm", C.c_int32), ("ared_guard", C.c_double),
        ("cauchy_norm", C.c_int32), ("pad1", C.c_int32),
    ]


class Counters(C.Structure):
    _fields_ = [
        ("outer", C.c_int64), ("accepted", C.c_int64), ("f_evals", C.c_int64),
        ("gh_evals", C.c_int64), ("cauchy_trials", C.c_int64), ("proj_trials", C.c_int64),
        ("cg_iters", C.c_int64), ("chol_calls", C.c_int64), ("subspace_passes", C.c_int64),
        ("sincos", C.c_int64), ("flops", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class Net(C.Structure):
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


class State(C.Structure):
    _fields_ = [(name, C.c_void_p) for name in (
        "br_x", "br_delta", "br_lam", "br_val", "br_tilde", "bus_w", "bus_th",
        "gen_pq", "gen_lam", "gen_tilde")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _load(_LIB_PATH)
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Run the oracle functions against another build of the C code (the tests use
    this to plant mistakes in a copy and check that the pins catch them)."""
    global _lib
    with _lock:
        old = _lib
        _lib = _load(path)
    try:
        yield
    finally:
        with _lock:
            _lib = old


def _load(path: str):
    if True:
        if True:
            L = C.CDLL(path)
            P = C.c_void_p
            L.ot_default_opts.argtypes = [C.POINTER(Opts)]
            L.ot_tron_solve.argtypes = [C.c_int, C.c_int, P, P, P, P, P, C.POINTER(Opts), P, P,
                                        P, C.POINTER(Counters)]
            L.ot_tron_solve.restype = C.c_int
            L.ot_tron_batch.argtypes = [C.c_int, C.c_int64, P, P, P, P, P, P, P, P,
                                        C.POINTER(Opts), P, P, P, P, C.c_int,
                                        C.POINTER(Counters)]
            L.ot_eval.argtypes = [C.c_int, C.c_int, P, P, P, P, P]
            L.ot_eval.restype = C.c_int
            L.ot_fscale.argtypes = [C.c_int, C.c_int, P, P]
            L.ot_fscale.restype = C.c_double
            L.ot_chol_left.argtypes = [C.c_int, P, C.c_int]
            L.ot_chol_left.restype = C.c_int
            L.ot_chol_shifted.argtypes = [C.c_int, P, P, C.c_double, C.c_int, P]
            L.ot_chol_shifted.restype = C.c_int
            L.ot_trqsol.argtypes = [C.c_int, P, P, C.c_double]
            L.ot_trqsol.restype = C.c_double
            L.ot_pgnorm.argtypes = [C.c_int, P, P, P, P]
            L.ot_pgnorm.restype = C.c_double
            L.ot_breakpt.argtypes = [C.c_int, P, P, P, P, P, P, P]
            L.ot_steihaug.argtypes = [C.c_int, P, P, P, C.c_double, C.c_double, C.c_int, P, P, P]
            L.ot_steihaug.restype = C.c_int
            L.ot_admm_init.argtypes = [C.POINTER(Net), C.POINTER(State)]
            L.ot_admm_run.argtypes = [C.POINTER(Net), C.POINTER(State), C.POINTER(Opts),
                                      C.c_int, C.c_int, P, P, P, C.POINTER(Counters)]
            L.ot_admm_branch_record.argtypes = [C.POINTER(Net), C.POINTER(State), C.c_int, P]
            L.ot_admm_phase_components.argtypes = [C.POINTER(Net), C.POINTER(State),
                                                   C.POINTER(Opts), C.c_int, P, P,
                                                   C.POINTER(Counters)]
            L.ot_admm_phase_buses.argtypes = [C.POINTER(Net), C.POINTER(State), P, P, P]
            L.ot_admm_mp_init.argtypes = [C.POINTER(MP)]
            L.ot_admm_mp_run.argtypes = [C.POINTER(MP), C.POINTER(Opts), C.c_int, C.c_int, P, P,
                                         C.POINTER(Counters)]
            L.ot_genramp_record.argtypes = [C.POINTER(MP), C.c_int, P]
            return L


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def default_opts(**over) -> Opts:
    o = Opts()
    lib().ot_default_opts(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def opts_dict(o: Opts) -> dict:
    return {name: getattr(o, name) for name, _ in Opts._fields_}


# ------------------------------------------------------------------------- TRON

def tron_solve(kind: int, params, l, u, x0, delta0: float = 1.0, opts: Opts | None = None):
    """Solve one problem; returns dict(x, f, pg, iters, status, delta, counters)."""
    o = opts or default_opts()
    params, l, u = _f64(params), _f64(l), _f64(u)
    x = _f64(x0).copy()
    n = x.size
    delta = np.array([delta0], dtype=np.float64)
    f = np.zeros(1)
    pg = np.zeros(1)
    it = np.zeros(1, dtype=np.int32)
    cnt = Counters()
    st = lib().ot_tron_solve(kind, n, _p(params), _p(l), _p(u), _p(x), _p(delta), C.byref(o),
                             _p(f), _p(pg), _p(it), C.byref(cnt))
    return dict(x=x, f=float(f[0]), pg=float(pg[0]), iters=int(it[0]), status=int(st),
                delta=float(delta[0]), counters=cnt.as_dict())


def tron_batch(kind: int, params, l, u, x0, delta0, n=None, opts: Opts | None = None,
               nthreads: int = 1):
    """Batch of problems.

    Uniform n: ``params`` [B, P], ``l, u, x0`` [B, n], ``delta0`` [B] or scalar.
    Uneven n: pass ``n`` (int array [B]) with ``params``, ``l``, ``u``, ``x0`` flat and
    concatenated in problem order (params of problem p: dense n^2 + 2n, branch 36,
    hs45 none).
    """
    o = opts or default_opts()
    x0 = np.asarray(x0, dtype=np.float64)
    if n is None:
        B, nn = x0.shape
        nvec = np.full(B, nn, dtype=np.int32)
        P = 0 if params is None else np.asarray(params).reshape(B, -1).shape[1]
        poff = (np.arange(B, dtype=np.int64) * P)
        voff = np.arange(B, dtype=np.int64) * nn
    else:
        nvec = np.ascontiguousarray(n, dtype=np.int32)
        B = nvec.size
        if kind == OBJ_DENSE:
            psz = nvec.astype(np.int64) ** 2 + 2 * nvec
        elif kind == OBJ_BRANCH:
            psz = np.full(B, 36, dtype=np.int64)
        else:
            psz = np.zeros(B, dtype=np.int64)
        poff = np.concatenate([[0], np.cumsum(psz)[:-1]]).astype(np.int64)
        voff = np.concatenate([[0], np.cumsum(nvec.astype(np.int64))[:-1]]).astype(np.int64)
    params = _f64(np.zeros(1) if params is None or np.size(params) == 0 else params).ravel()
    l = _f64(l).ravel()
    u = _f64(u).ravel()
    x = _f64(x0).ravel().copy()
    delta = np.broadcast_to(np.asarray(delta0, dtype=np.float64), (B,)).copy()
    f = np.zeros(B)
    pg = np.zeros(B)
    it = np.zeros(B, dtype=np.int32)
    st = np.zeros(B, dtype=np.int32)
    cnt = Counters()
    lib().ot_tron_batch(kind, B, _p(nvec), _p(poff), _p(voff), _p(params), _p(l), _p(u), _p(x),
                        _p(delta), C.byref(o), _p(f), _p(pg), _p(it), _p(st), int(nthreads),
                        C.byref(cnt))
    if n is None:
        x = x.reshape(B, -1)
    return dict(x=x, f=f, pg=pg, iters=it, status=st, delta=delta, counters=cnt.as_dict())


def eval_obj(kind: int, params, x):
    """f, gradient and Hessian of one objective at x."""
    x = _f64(x)
    n = x.size
    params = _f64(np.zeros(1) if params is None else params)
    f = np.zeros(1)
    g = np.zeros(n)
    H = np.zeros((n, n))
    r = lib().ot_eval(kind, n, _p(params), _p(x), _p(f), _p(g), _p(H))
    if r != 0:
        raise ValueError("bad objective kind / size")
    return float(f[0]), g, H


def fscale(kind: int, params, x) -> float:
    """The rounding scale S of f at x that guards the reduction ratio: the sum of the
    magnitudes of the terms f is assembled from."""
    x = _f64(x)
    params = _f64(np.zeros(1) if params is None else params)
    return float(lib().ot_fscale(kind, x.size, _p(params), _p(x)))


def chol(A):
    """Left-looking Cholesky; returns the lower factor or None if not positive definite."""
    A = _f64(A).copy()
    m = A.shape[0]
    r = lib().ot_chol_left(m, _p(A), m)
    return None if r else np.tril(A)


def chol_shifted(A, shift_frac=1e-3, max_shift=30):
    """Shifted Cholesky; returns (L_with_mirrored_upper, alpha) or (None, None)."""
    A = _f64(A)
    m = A.shape[0]
    L = np.zeros((m, m))
    a = np.zeros(1)
    r = lib().ot_chol_shifted(m, _p(A), _p(L), shift_frac, max_shift, _p(a))
    return (None, None) if r else (L, float(a[0]))


def trqsol(x, p, delta):
    x, p = _f64(x), _f64(p)
    return lib().ot_trqsol(x.size, _p(x), _p(p), float(delta))


def pgnorm(x, g, l, u):
    x, g, l, u = _f64(x), _f64(g), _f64(l), _f64(u)
    return lib().ot_pgnorm(x.size, _p(x), _p(g), _p(l), _p(u))


def breakpt(x, w, l, u):
    x, w, l, u = _f64(x), _f64(w), _f64(l), _f64(u)
    nb = np.zeros(1, dtype=np.int32)
    bmin = np.zeros(1)
    bmax = np.zeros(1)
    lib().ot_breakpt(x.size, _p(x), _p(w), _p(l), _p(u), _p(nb), _p(bmin), _p(bmax))
    return int(nb[0]), float(bmin[0]), float(bmax[0])


def steihaug(A, L, bhat, delta, rtol=0.1, norm=0, with_len=False):
    """Steihaug PCG; returns (w, info, iterations) or, with ``with_len``, also the
    step's length in the bounded norm (||s|| for norm 0, ||w|| for norm 1)."""
    A, L, bhat = _f64(A), _f64(L), _f64(bhat)
    m = bhat.size
    s = np.zeros(m)
    it = np.zeros(1, dtype=np.int32)
    tl = np.zeros(1)
    info = lib().ot_steihaug(m, _p(A), _p(L), _p(bhat), float(delta), float(rtol), int(norm),
                             _p(s), _p(it), _p(tl))
    if with_len:
        return s, int(info), int(it[0]), float(tl[0])
    return s, int(info), int(it[0])


# ------------------------------------------------------------------------- ADMM

class Admm:
    """Oracle ADMM instance over a network dict (see paper_2106_14995_gb300.synth)."""

    def __init__(self, net: dict, rho: float = 400.0, rho_line: float | None = None,
                 vmin: float = 0.9, vmax: float = 1.1):
        self._keep = {}

        def keep(name, a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep[name] = a
            return a.ctypes.data

        c = Net()
        c.nbus = int(net["nbus"])
        c.nbranch = int(len(net["br_from"]))
        c.ngen = int(len(net["gen_bus"]))
        c.br_from = keep("br_from", net["br_from"], np.int32)
        c.br_to = keep("br_to", net["br_to"], np.int32)
        c.br_coef = keep("br_coef", net["br_coef"], np.float64)
        c.br_smax2 = keep("br_smax2", net["br_smax2"], np.float64)
        c.gen_bus = keep("gen_bus", net["gen_bus"], np.int32)
        for k in ("gen_c2", "gen_c1", "gen_pmin", "gen_pmax", "gen_qmin", "gen_qmax",
                  "bus_pd", "bus_qd", "bus_gsh", "bus_bsh"):
            setattr(c, k, keep(k, net[k], np.float64))
        c.rho = float(rho)
        c.rho_line = float(rho if rho_line is None else rho_line)
        c.vmin = float(vmin)
        c.vmax = float(vmax)
        self.net = c
        nb, nl, ng = c.nbus, c.nbranch, c.ngen
        self.arrays = dict(
            br_x=np.zeros((nl, 4)), br_delta=np.zeros(nl), br_lam=np.zeros((nl, 8)),
            br_val=np.zeros((nl, 8)), br_tilde=np.zeros((nl, 4)), bus_w=np.zeros(nb),
            bus_th=np.zeros(nb), gen_pq=np.zeros((ng, 2)), gen_lam=np.zeros((ng, 2)),
            gen_tilde=np.zeros((ng, 2)))
        self.state = State(**{k: v.ctypes.data for k, v in self.arrays.items()})
        lib().ot_admm_init(C.byref(self.net), C.byref(self.state))
        self.counters = Counters()
        self.status_counts = np.zeros(6, dtype=np.int64)

    def run(self, niters: int, opts: Opts | None = None, nthreads: int = 1):
        o = opts or default_opts()
        hp = np.zeros(niters)
        hd = np.zeros(niters)
        lib().ot_admm_run(C.byref(self.net), C.byref(self.state), C.byref(o), int(niters),
                          int(nthreads), _p(hp), _p(hd), _p(self.status_counts),
                          C.byref(self.counters))
        return hp, hd

    def phase_components(self, gen_mask, br_mask, opts: Opts | None = None,
                         nthreads: int = 1) -> None:
        """Generator and branch updates of the masked components (one phase of the
        iteration, as a partitioned run performs it)."""
        o = opts or default_opts()
        gm = np.ascontiguousarray(gen_mask, dtype=np.uint8)
        bm = np.ascontiguousarray(br_mask, dtype=np.uint8)
        lib().ot_admm_phase_components(C.byref(self.net), C.byref(self.state), C.byref(o),
                                       int(nthreads), _p(gm), _p(bm), C.byref(self.counters))

    def phase_buses(self, bus_mask):
        """Bus updates of the masked buses with the multipliers of their pairs; returns
        the squared primal and (unscaled) dual residual sums of those pairs."""
        bm = np.ascontiguousarray(bus_mask, dtype=np.uint8)
        pr2 = np.zeros(1)
        du2 = np.zeros(1)
        lib().ot_admm_phase_buses(C.byref(self.net), C.byref(self.state), _p(bm), _p(pr2),
                                  _p(du2))
        return float(pr2[0]), float(du2[0])

    def branch_record(self, k: int) -> np.ndarray:
        rec = np.zeros(36)
        lib().ot_admm_branch_record(C.byref(self.net), C.byref(self.state), int(k), _p(rec))
        return rec


# ----------------------------------------------------------- multi-period ADMM

class MP(C.Structure):
    _fields_ = [("T", C.c_int32), ("nets", C.c_void_p), ("states", C.c_void_p),
                ("ramp", C.c_void_p), ("rho_ramp", C.c_double), ("gen_delta", C.c_void_p)]


class MultiPeriodAdmm:
    """Oracle multi-period ADMM: T periods of ``net`` with loads scaled by
    ``load_scale[t]``, generators coupled across periods by the ramp penalty
    rho_ramp/2 max(0, |p_t - p_{t-1}| - ramp[g])^2 (``ramp`` scalar or [ngen])."""

    def __init__(self, net: dict, load_scale, ramp, rho_ramp: float = 400.0,
                 rho: float = 400.0, rho_line: float | None = None, vmin: float = 0.9,
                 vmax: float = 1.1):
        self.T = T = len(load_scale)
        ng = len(net["gen_bus"])
        self.periods = []
        for t in range(T):
            nt = dict(net)
            nt["bus_pd"] = np.asarray(net["bus_pd"], dtype=np.float64) * float(load_scale[t])
            nt["bus_qd"] = np.asarray(net["bus_qd"], dtype=np.float64) * float(load_scale[t])
            self.periods.append(Admm(nt, rho=rho, rho_line=rho_line, vmin=vmin, vmax=vmax))
        self._nets = (Net * T)(*[a.net for a in self.periods])
        self._states = (State * T)(*[a.state for a in self.periods])
        self.ramp = np.ascontiguousarray(np.broadcast_to(np.asarray(ramp, dtype=np.float64),
                                                         (ng,)))
        self.gen_delta = np.zeros(ng)
        self.mp = MP(T=T, nets=C.cast(self._nets, C.c_void_p).value,
                     states=C.cast(self._states, C.c_void_p).value,
                     ramp=self.ramp.ctypes.data, rho_ramp=float(rho_ramp),
                     gen_delta=self.gen_delta.ctypes.data)
        lib().ot_admm_mp_init(C.byref(self.mp))
        self.counters = Counters()

    def run(self, niters: int, opts: Opts | None = None, nthreads: int = 1):
        o = opts or default_opts()
        hp = np.zeros(niters)
        hd = np.zeros(niters)
        lib().ot_admm_mp_run(C.byref(self.mp), C.byref(o), int(niters), int(nthreads),
                             _p(hp), _p(hd), C.byref(self.counters))
        return hp, hd

    def genramp_record(self, g: int) -> np.ndarray:
        rec = np.zeros(8 + 2 * self.T)
        lib().ot_genramp_record(C.byref(self.mp), int(g), _p(rec))
        return rec

    def state(self, t: int) -> dict:
        return self.periods[t].arrays
