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

    # ---- host-buffer path: arrays in (page-locked) host memory, copies by the library
    def host_enable(self) -> None:
        """Allocate the two device buffer sets of the host-buffer path (setup time)."""
        nt.check(self._lib.tron_batch_host_enable(self._h), "tron_batch_host_enable")

    def solve_host(self, params, lower, upper, x0, delta0, out: dict) -> dict:
        """Enqueue one solve of host arrays (torch CPU tensors, pinned for overlap); the
        results land in ``out`` (x, delta, f, pg, iters, status host tensors) once
        ``host_sync`` returns.  Inputs may be shared by calls in flight; results are
        copied out in call order."""
        hp = nt.hptr
        nt.check(self._lib.tron_batch_solve_host(
            self._h, hp(params), hp(lower), hp(upper), hp(x0), hp(delta0), hp(out["x"]),
            hp(out["delta"]), hp(out["f"]), hp(out["pg"]), hp(out["iters"]),
            hp(out["status"])), "tron_batch_solve_host")
        return out

    def host_sync(self) -> None:
        nt.check(self._lib.tron_batch_host_sync(self._h), "tron_batch_host_sync")

    def host_outputs(self, total_n: int, pin: bool = True) -> dict:
        """A set of host result tensors for solve_host (total_n = length of x)."""
        B = self.nprob
        mk = lambda n, dt: torch.empty(n, dtype=dt).pin_memory() if pin else \
            torch.empty(n, dtype=dt)
        return dict(x=mk(total_n, torch.float64), delta=mk(B, torch.float64),
                    f=mk(B, torch.float64), pg=mk(B, torch.float64),
                    iters=mk(B, torch.int32), status=mk(B, torch.int32))

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


OP_LATENCY_NAMES = ("fp64 fma", "fp64 add", "fp64 max", "fp64 compare+select",
                    "int64 compare+select", "solver quotient", "ieee division",
                    "solver square root", "ieee sqrt", "library sin", "sine series",
                    "reciprocal estimate", "64-bit shuffle", "library cos", "library sincos",
                    "fp32 fma")


def op_latency(op: int, lanes: int = 32, stream=None) -> float:
    """SM cycles per dependent operation of kind ``op`` (see OP_LATENCY_NAMES) with
    ``lanes`` active threads in one CTA (tron_bench_op_latency)."""
    lib = nt.load()
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    nt.check(lib.tron_bench_op_latency(int(op), int(lanes), out.data_ptr(),
                                       nt.stream_handle(stream)), "tron_bench_op_latency")
    torch.cuda.synchronize()
    return float(out.item()) / float(lib.tron_bench_op_chain())
