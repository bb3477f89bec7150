"""Continuous-batching server of independent ADMM instances on one GPU.

Requests (networks with arrival times) are admitted into a resident ``AdmmPool`` as soon
as they have arrived and the pool has free slot ranges (the pool's capacity is the
device-memory budget; a request that does not fit waits, first come first served).
Every live instance advances in the same launches; after each chunk of iterations the
latest residuals of all instances are read back (one small copy) and the instances that
reached ``primal <= tol and dual <= tol``, or the iteration cap, are retired and their
slots freed.  Per-instance arithmetic does not depend on the other residents (see
``AdmmPool``), so every result equals the instance's run alone.

``serial_plain`` runs the same requests one after another, each alone in its own
single-network ADMM, as the baseline the served latencies are compared with.
"""
from __future__ import annotations

import collections
import time

import numpy as np
import torch

from .admm import Admm, AdmmPool


def percentile(v, q):
    return float(np.percentile(np.asarray(v, dtype=np.float64), q)) if len(v) else float("nan")


class AdmmServer:
    """``pool``: an object with the ``AdmmPool`` calls the loop uses (add, step,
    residuals, remove, get_state, close); by default a new ``AdmmPool`` of the given
    capacities."""

    def __init__(self, cap_bus: int, cap_branch: int, cap_gen: int, cap_instances: int,
                 chunk: int = 8, tol: float = 1e-4, max_iters: int = 20000,
                 history_len: int = 256, opts=None, pool=None):
        self.pool = pool if pool is not None else AdmmPool(cap_bus, cap_branch, cap_gen,
                                                           cap_instances, history_len, opts)
        self.chunk = int(chunk)
        self.tol = float(tol)
        self.max_iters = int(max_iters)

    def run(self, requests, clock=time.perf_counter, keep_state: bool = False):
        """requests: list of dict(t=arrival offset in s, net=network dict, id=..., and
        optionally rho, the instance's penalty).  Returns one record per request:
        arrival, admitted, finished (s from the start), iterations, residuals,
        converged."""
        pending = collections.deque(sorted(requests, key=lambda r: r["t"]))
        live = {}
        done = []
        steps = 0
        t0 = clock()
        while pending or live:
            now = clock() - t0
            while pending and pending[0]["t"] <= now:
                req0 = pending[0]
                inst = (self.pool.add(req0["net"], rho=req0["rho"]) if "rho" in req0
                        else self.pool.add(req0["net"]))
                if inst is None:
                    break  # no room until some instance retires
                req = pending.popleft()
                live[inst] = dict(req=req, admitted=now)
            if not live:
                if pending:
                    time.sleep(max(0.0, min(0.002, pending[0]["t"] - (clock() - t0))))
                continue
            self.pool.step(self.chunk)
            steps += 1
            it, pr, du = self.pool.residuals()
            now = clock() - t0
            for inst in list(live):
                conv = bool(pr[inst] <= self.tol and du[inst] <= self.tol)
                if conv or it[inst] >= self.max_iters:
                    rec = live.pop(inst)
                    out = dict(id=rec["req"].get("id"), arrival=rec["req"]["t"],
                               admitted=rec["admitted"], finished=now, iterations=int(it[inst]),
                               primal=float(pr[inst]), dual=float(du[inst]), converged=conv,
                               nbus=int(rec["req"]["net"]["nbus"]))
                    if keep_state:
                        out["state"] = self.pool.get_state(inst)
                    done.append(out)
                    self.pool.remove(inst)
        self.launch_steps = steps
        return done

    def close(self):
        self.pool.close()


def serial_plain(requests, chunk: int = 8, tol: float = 1e-4, max_iters: int = 20000,
                 clock=time.perf_counter):
    """Each request alone in a single-network ADMM, in arrival order (FIFO): measured
    service times, latencies from a FIFO queue over the arrival times."""
    out = []
    t_free = 0.0
    for req in sorted(requests, key=lambda r: r["t"]):
        a = Admm(req["net"], rho=req.get("rho", 400.0))
        torch.cuda.synchronize()
        s0 = clock()
        its, conv = 0, False
        pr = du = float("nan")
        while its < max_iters:
            pr, du = a.step(chunk)
            its += chunk
            if pr <= tol and du <= tol:
                conv = True
                break
        service = clock() - s0
        a.close()
        start = max(req["t"], t_free)
        t_free = start + service
        out.append(dict(id=req.get("id"), arrival=req["t"], finished=t_free, iterations=its,
                        primal=pr, dual=du, converged=conv, service=service,
                        nbus=int(req["net"]["nbus"])))
    return out


def summarize(records) -> dict:
    """Latency percentiles over all records (for instances that hit the iteration cap,
    the time to the cap) and over the converged ones alone (time to solution)."""
    lat = [r["finished"] - r["arrival"] for r in records]
    lat_c = [r["finished"] - r["arrival"] for r in records if r["converged"]]
    its = sum(r["iterations"] for r in records)
    span = (max(r["finished"] for r in records) - min(r["arrival"] for r in records)
            if records else float("nan"))
    return dict(instances=len(records), p50_s=percentile(lat, 50), p99_s=percentile(lat, 99),
                mean_s=float(np.mean(lat)) if lat else float("nan"),
                p50_converged_s=percentile(lat_c, 50), p99_converged_s=percentile(lat_c, 99),
                iterations=int(its), makespan_s=span,
                agg_iters_per_s=its / span if span and span > 0 else float("nan"),
                converged=int(sum(r["converged"] for r in records)))
