"""Batched TRON on the GPU: a thin object wrapper over the tron_batch_* C ABI."""
from __future__ import annotations

import ctypes as C

import torch

from . import native as nt

STATUS_NAMES = ["CONVERGED", "MAX_ITER", "TR_TOO_SMALL", "CHOL_FAIL", "NONFINITE",
                "BAD_BOUNDS"]


def options(**over) -> nt.TronOptions:
    o = nt.tron_options_default()
    for k, v in over.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class TronBatch:
    """A batch of problems of one objective family.

    ``n``: uniform size, or ``n_list``: per-problem sizes (records and vectors of
    consecutive problems concatenated).  Buffers are torch CUDA float64 tensors.
    """

    def __init__(self, kind: int, nprob: int, n: int | None = None, n_list=None,
                 opts: nt.TronOptions | None = None, stream=None):
        self._lib = nt.load()
        self.kind = int(kind)
        self.nprob = int(nprob)
        self.opts = opts or nt.tron_options_default()
        h = C.c_void_p()
        if n_list is not None:
            arr = (C.c_int32 * self.nprob)(*[int(v) for v in n_list])
            nptr = C.cast(arr, C.c_void_p)
            nu = 0
        else:
            nptr = None
            nu = int(n)
        nt.check(self._lib.tron_batch_create(C.byref(h), self.kind, self.nprob, nptr, nu,
                                             C.byref(self.opts), nt.stream_handle(stream)),
                 "tron_batch_create")
        self._h = h

    def set_options(self, opts: nt.TronOptions) -> None:
        nt.check(self._lib.tron_batch_set_options(self._h, C.byref(opts)),
                 "tron_batch_set_options")
        self.opts = opts

    def solve(self, params, lower, upper, x, delta, f=None, pg=None, iters=None,
              status=None, stream=None) -> dict:
        dev = x.device
        B = self.nprob
        f = f if f is not None else torch.empty(B, dtype=torch.float64, device=dev)
        pg = pg if pg is not None else torch.empty(B, dtype=torch.float64, device=dev)
        iters = iters if iters is not None else torch.empty(B, dtype=torch.int32, device=dev)
        status = status if status is not None else torch.empty(B, dtype=torch.int32,
                                                                device=dev)
        nt.check(self._lib.tron_batch_solve(
            self._h, nt.ptr(params), nt.ptr(lower), nt.ptr(upper), nt.ptr(x), nt.ptr(delta),
            nt.ptr(f), nt.ptr(pg), nt.ptr(iters), nt.ptr(status), nt.stream_handle(stream)),
            "tron_batch_solve")
        return dict(x=x, delta=delta, f=f, pg=pg, iters=iters, status=status)

    def autotune(self, params, lower, upper, x0, delta0, sample: int = 8192,
                 stream=None) -> list:
        """Time every kernel variant per size class on a sample; keep the fastest."""
        nt.check(self._lib.tron_batch_autotune(
            self._h, nt.ptr(params), nt.ptr(lower), nt.ptr(upper), nt.ptr(x0), nt.ptr(delta0),
            int(sample), nt.stream_handle(stream)), "tron_batch_autotune")
        return self.choices()

    def choices(self) -> list:
        out = []
        for bi in range(int(self._lib.tron_batch_buckets(self._h))):
            v = [C.c_int32() for _ in range(4)]
            cnt = C.c_int64()
            nt.check(self._lib.tron_batch_get_choice(self._h, bi, *[C.byref(x) for x in v],
                                                     C.byref(cnt)), "tron_batch_get_choice")
            out.append(dict(N=v[0].value, group=v[1].value, layout=v[2].value,
                            warps_per_block=v[3].value, count=cnt.value))
        return out

    @property
    def last_launches(self) -> int:
        return int(self._lib.tron_batch_last_launches(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.tron_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
