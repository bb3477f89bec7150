"""Component ADMM on the GPU (Sec. 6.1): thin wrappers over the admm_* / admm_pool_* /
admm_mp_* ABI.

``Admm`` holds one network; ``AdmmPool`` holds many independent instances resident on
the device and advances them together (continuous batching); ``AdmmMultiPeriod`` holds T
periods of one network coupled by generator ramp limits.  Networks are dicts as produced
by ``synth.network`` (host numpy arrays); they are copied to the device.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import native as nt

STATE_SHAPES = dict(br_x=("nbranch", 4), br_delta=("nbranch",), br_lam=("nbranch", 8),
                    br_val=("nbranch", 8), br_tilde=("nbranch", 4), bus_w=("nbus",),
                    bus_th=("nbus",), gen_pq=("ngen", 2), gen_lam=("ngen", 2),
                    gen_tilde=("ngen", 2))


class _NetHolder:
    """Keeps the contiguous host arrays of a network alive while C reads them."""

    def __init__(self, net: dict, rho: float, rho_line: float | None, vmin: float, vmax: float):
        keep = {}

        def arr(name, dtype):
            a = np.ascontiguousarray(net[name], dtype=dtype)
            keep[name] = a
            return a.ctypes.data

        s = nt.AdmmNetwork()
        s.nbus = int(net["nbus"])
        s.nbranch = int(len(net["br_from"]))
        s.ngen = int(len(net["gen_bus"]))
        s.br_from = arr("br_from", np.int32)
        s.br_to = arr("br_to", np.int32)
        s.br_coef = arr("br_coef", np.float64)
        s.br_smax2 = arr("br_smax2", np.float64)
        s.gen_bus = arr("gen_bus", np.int32)
        for k in ("gen_c2", "gen_c1", "gen_pmin", "gen_pmax", "gen_qmin", "gen_qmax",
                  "bus_pd", "bus_qd", "bus_gsh", "bus_bsh"):
            setattr(s, k, arr(k, np.float64))
        s.rho = float(rho)
        s.rho_line = float(rho if rho_line is None else rho_line)
        s.vmin = float(vmin)
        s.vmax = float(vmax)
        self.s = s
        self.keep = keep
        self.sizes = dict(nbus=s.nbus, nbranch=s.nbranch, ngen=s.ngen)


def _state_buffers(sizes: dict) -> dict:
    return {k: np.zeros(tuple(sizes[d] if isinstance(d, str) else d for d in shp))
            for k, shp in STATE_SHAPES.items()}


def _view(bufs: dict, iteration: int = 0) -> nt.AdmmStateView:
    v = nt.AdmmStateView(**{k: bufs[k].ctypes.data for k in STATE_SHAPES})
    v.iteration = int(iteration)
    return v


class Admm:
    """One network on the GPU; ``step(n)`` runs n iterations (replayed CUDA graph)."""

    def __init__(self, net: dict, rho: float = 400.0, rho_line: float | None = None,
                 vmin: float = 0.9, vmax: float = 1.1, opts: nt.TronOptions | None = None,
                 stream=None):
        self._lib = nt.load()
        self._net = _NetHolder(net, rho, rho_line, vmin, vmax)
        self.sizes = self._net.sizes
        h = C.c_void_p()
        nt.check(self._lib.admm_create(C.byref(h), C.byref(self._net.s),
                                       C.byref(opts) if opts is not None else None,
                                       nt.stream_handle(stream)), "admm_create")
        self._h = h
        self.stream = stream

    def step(self, n_iters: int, residuals: bool = True):
        pr = C.c_double()
        du = C.c_double()
        nt.check(self._lib.admm_step(self._h, int(n_iters),
                                     C.byref(pr) if residuals else None,
                                     C.byref(du) if residuals else None,
                                     nt.stream_handle(self.stream)), "admm_step")
        return (pr.value, du.value) if residuals else None

    def history(self, first: int, count: int):
        hp = np.zeros(count)
        hd = np.zeros(count)
        nt.check(self._lib.admm_residual_history(self._h, int(first), int(count),
                                                 hp.ctypes.data, hd.ctypes.data,
                                                 nt.stream_handle(self.stream)),
                 "admm_residual_history")
        return hp, hd

    @property
    def iterations(self) -> int:
        return int(self._lib.admm_iterations(self._h))

    @property
    def branch_group(self) -> int:
        """Lanes per branch problem in the branch launch (1, 2 or 4)."""
        return int(self._lib.admm_pool_branch_group(self._h))

    @property
    def launches_per_iteration(self) -> int:
        """GPU kernel launches of one iteration: 2, or 3 when one-lane branch solves
        are finished on four lanes (options.split_outer > 0)."""
        return int(self._lib.admm_pool_launches_per_iteration(self._h))

    def get_state(self) -> dict:
        bufs = _state_buffers(self.sizes)
        v = _view(bufs)
        nt.check(self._lib.admm_get_state(self._h, C.byref(v), nt.stream_handle(self.stream)),
                 "admm_get_state")
        bufs["iteration"] = v.iteration
        return bufs

    def set_state(self, state: dict) -> None:
        bufs = {k: np.ascontiguousarray(state[k], dtype=np.float64) for k in STATE_SHAPES}
        v = _view(bufs, state.get("iteration", 0))
        nt.check(self._lib.admm_set_state(self._h, C.byref(v), nt.stream_handle(self.stream)),
                 "admm_set_state")

    def branch_status_counts(self) -> np.ndarray:
        c = np.zeros(6, dtype=np.int64)
        nt.check(self._lib.admm_branch_status_counts(self._h, c.ctypes.data,
                                                     nt.stream_handle(self.stream)),
                 "admm_branch_status_counts")
        return c

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.admm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AdmmPool:
    """Resident pool of independent ADMM instances sharing every launch."""

    def __init__(self, cap_bus: int, cap_branch: int, cap_gen: int, cap_instances: int,
                 history_len: int = 4096, opts: nt.TronOptions | None = None, stream=None):
        self._lib = nt.load()
        h = C.c_void_p()
        nt.check(self._lib.admm_pool_create(C.byref(h), int(cap_bus), int(cap_branch),
                                            int(cap_gen), int(cap_instances), int(history_len),
                                            C.byref(opts) if opts is not None else None,
                                            nt.stream_handle(stream)), "admm_pool_create")
        self._h = h
        self.cap_instances = int(cap_instances)
        self.stream = stream
        self._nets = {}

    def add(self, net: dict, rho: float = 400.0, rho_line: float | None = None,
            vmin: float = 0.9, vmax: float = 1.1):
        """Admit an instance; returns its id, or None when the pool has no room."""
        holder = _NetHolder(net, rho, rho_line, vmin, vmax)
        i = C.c_int32(-1)
        rc = self._lib.admm_pool_add(self._h, C.byref(holder.s), C.byref(i),
                                     nt.stream_handle(self.stream))
        if rc == 2:  # TRON_ENOMEM: no free slots now
            return None
        nt.check(rc, "admm_pool_add")
        self._nets[i.value] = holder
        return i.value

    def remove(self, inst: int) -> None:
        nt.check(self._lib.admm_pool_remove(self._h, int(inst), nt.stream_handle(self.stream)),
                 "admm_pool_remove")
        self._nets.pop(inst, None)

    def step(self, n_iters: int) -> None:
        nt.check(self._lib.admm_pool_step(self._h, int(n_iters), nt.stream_handle(self.stream)),
                 "admm_pool_step")

    def residuals(self):
        it = np.zeros(self.cap_instances, dtype=np.int64)
        pr = np.zeros(self.cap_instances)
        du = np.zeros(self.cap_instances)
        nt.check(self._lib.admm_pool_residuals(self._h, it.ctypes.data, pr.ctypes.data,
                                               du.ctypes.data, nt.stream_handle(self.stream)),
                 "admm_pool_residuals")
        return it, pr, du

    def history(self, inst: int, first: int, count: int):
        hp = np.zeros(count)
        hd = np.zeros(count)
        nt.check(self._lib.admm_pool_history(self._h, int(inst), int(first), int(count),
                                             hp.ctypes.data, hd.ctypes.data,
                                             nt.stream_handle(self.stream)),
                 "admm_pool_history")
        return hp, hd

    def get_state(self, inst: int) -> dict:
        bufs = _state_buffers(self._nets[inst].sizes)
        v = _view(bufs)
        nt.check(self._lib.admm_pool_get_state(self._h, int(inst), C.byref(v),
                                               nt.stream_handle(self.stream)),
                 "admm_pool_get_state")
        bufs["iteration"] = v.iteration
        return bufs

    @property
    def live(self) -> int:
        return int(self._lib.admm_pool_live(self._h))

    @property
    def branch_group(self) -> int:
        """Lanes per branch problem in the branch launch (1, 2 or 4)."""
        return int(self._lib.admm_pool_branch_group(self._h))

    @property
    def launches_per_iteration(self) -> int:
        """GPU kernel launches of one iteration: 2, or 3 when one-lane branch solves
        are finished on four lanes (options.split_outer > 0)."""
        return int(self._lib.admm_pool_launches_per_iteration(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.admm_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AdmmMultiPeriod:
    """T periods of one network (loads scaled by ``load_scale[t]``) coupled by generator
    ramp limits ``ramp`` (scalar or [ngen]) through the penalty ``rho_ramp``; see
    admm_mp_create in include/admm.h."""

    def __init__(self, net: dict, load_scale, ramp, rho_ramp: float = 400.0,
                 rho: float = 400.0, rho_line: float | None = None, vmin: float = 0.9,
                 vmax: float = 1.1, opts: nt.TronOptions | None = None, stream=None):
        self._lib = nt.load()
        self._net = _NetHolder(net, rho, rho_line, vmin, vmax)
        self.sizes = self._net.sizes
        self.T = len(load_scale)
        self._scale = np.ascontiguousarray(load_scale, dtype=np.float64)
        self._ramp = np.ascontiguousarray(
            np.broadcast_to(np.asarray(ramp, dtype=np.float64), (self.sizes["ngen"],)))
        h = C.c_void_p()
        nt.check(self._lib.admm_mp_create(C.byref(h), C.byref(self._net.s), int(self.T),
                                          self._scale.ctypes.data, self._ramp.ctypes.data,
                                          float(rho_ramp),
                                          C.byref(opts) if opts is not None else None,
                                          nt.stream_handle(stream)), "admm_mp_create")
        self._h = h
        self.stream = stream

    @property
    def launches_per_iteration(self) -> int:
        """GPU kernel launches of one iteration: the periods' branch launch (and its
        four-lane continuation), the generator chains with their gather and scatter, and
        the bus launch."""
        return int(self._lib.admm_mp_launches_per_iteration(self._h))

    def step(self, n_iters: int, residuals: bool = True):
        pr = C.c_double()
        du = C.c_double()
        nt.check(self._lib.admm_mp_step(self._h, int(n_iters),
                                        C.byref(pr) if residuals else None,
                                        C.byref(du) if residuals else None,
                                        nt.stream_handle(self.stream)), "admm_mp_step")
        return (pr.value, du.value) if residuals else None

    def get_state(self, period: int) -> dict:
        bufs = _state_buffers(self.sizes)
        v = _view(bufs)
        nt.check(self._lib.admm_mp_get_state(self._h, int(period), C.byref(v),
                                             nt.stream_handle(self.stream)),
                 "admm_mp_get_state")
        bufs["iteration"] = v.iteration
        return bufs

    def gen_status_counts(self) -> np.ndarray:
        c = np.zeros(6, dtype=np.int64)
        nt.check(self._lib.admm_mp_gen_status_counts(self._h, c.ctypes.data,
                                                     nt.stream_handle(self.stream)),
                 "admm_mp_gen_status_counts")
        return c

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.admm_mp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
