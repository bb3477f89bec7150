"""Benchmark: batched TRON subproblems/s at a 1e-6 projected-gradient tolerance.

Workload (the configuration the headline metric is quoted on): 10,000 dense problems,
n = 32, f = 1/2 x'Qx + c'x + 0.1 sum x^4, Q = U diag(lam) U' with U Haar and lam
log-uniform in [1, 1e3], c ~ N(0, 4^2), l ~ U[-2, -0.5], u ~ U[0.5, 2], x0 = 0, FP64.
One step = one batched solve of the whole batch from x0 (one kernel launch).

Launch:  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
         (N > 1 under torch.distributed.run: each rank solves its own batch; weak scaling)

Timed region: K steps bracketed by a barrier and device synchronisation; device time
from CUDA events on the launch stream; max over ranks.  Inputs larger than L2: each
step reads its own copy of the batch (rotating buffers, total > 2 x L2).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TRON subproblems/s & ADMM iters/s at 1e-6 proj-grad; serving p50/p99 vs plain"
UNIT = "subproblems/s"
B_DEFAULT = 10000
N_VARS = 32
L2_BYTES = 129 * 2 ** 20
FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2.070  # 2 DFMA/clk/SM x 2 flop x 152 SMs x 2.07 GHz
# algorithmic bytes of one n = 32 problem: record (Q, c, d), l, u, x0, delta in; x,
# delta, f, pg (FP64) and iterations, status (int32) out
ALG_BYTES_PER_PROBLEM = (8 * (N_VARS * N_VARS + 2 * N_VARS) + 3 * 8 * N_VARS + 8 +
                         8 * N_VARS + 3 * 8 + 2 * 4)


def hbm_peak_gbs():
    """Measured copy bandwidth of this GPU model (MEASURED_PEAKS.json), else the
    fallback of an earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"
# From one ncu capture of the timed kernel (profiles/tron_dense32_n10000.md, 2,000
# problems, scaled per problem to the launch), valid only for the kernel sources it was
# taken on: DRAM bytes (19.08 MB per 2,000 problems) and the FP64 flops the kernel
# executes (thread-level DFMA x 2 + DADD + DMUL: 301.2 Mflop per 2,000 problems).
TRAFFIC_BYTES_PER_PROBLEM = 19.08224e6 / 2000
EXEC_FLOPS_PER_PROBLEM = (2 * 128374664 + 25437882 + 19049401) / 2000
TRAFFIC_SOURCES_SHA1 = "8e6fa49cc7411b1a5bc59df4c7610f5843bd5ba9"
TRAFFIC_SOURCES = ("tron_common.cuh", "tron_objectives.cuh", "tron_solver.cuh")


def _sources_match() -> bool:
    import hashlib
    h = hashlib.sha1()
    for name in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2106_14995_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest() == TRAFFIC_SOURCES_SHA1


def traffic_per_launch(nprob: int):
    """DRAM bytes of one launch, or None when the kernel changed since the capture."""
    return TRAFFIC_BYTES_PER_PROBLEM * nprob if _sources_match() else None


def executed_flops_per_launch(nprob: int):
    """FP64 flops the kernel executes per launch, or None when it changed since."""
    return EXEC_FLOPS_PER_PROBLEM * nprob if _sources_match() else None


def fp64_peak_measured(dev, lib):
    """FP64 FMA throughput of this GPU measured with the library's probe (8 independent
    FMA chains per thread, 8 CTAs of 256 threads per SM): the median of five launches of
    about 10 ms, in GFLOP/s."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads, iters = 8 * sms, 256, 4000
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev)
    ts = []
    for rep in range(7):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rc = lib.tron_bench_fp64_fma(out.data_ptr(), blocks, threads, iters, st.cuda_stream)
        e1.record(st)
        torch.cuda.synchronize(dev)
        if rc != 0:
            return None
        if rep >= 2:
            ts.append(e0.elapsed_time(e1))
    flops = 16.0 * iters * blocks * threads
    return flops / (float(np.median(ts)) * 1e-3) / 1e9


def fp64_roofline(flops, seconds, peak_measured, kernel, extra=None):
    """An "alu" roofline block: oracle-counted FP64 flops over device time, against the
    nominal FP64 peak (2 DFMA/clk/SM x 152 SMs x 2.07 GHz) and the probe's measured one."""
    achieved = flops / seconds / 1e9
    r = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
         "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
         "peak_measured": peak_measured,
         "frac_measured": (achieved / peak_measured) if peak_measured else None}
    if extra:
        r.update(extra)
    return r


def hbm_block(nbytes, seconds):
    peak, src = hbm_peak_gbs()
    a = nbytes / seconds / 1e9
    return {"achieved": a, "peak": peak, "peak_source": src, "unit": "GB/s", "frac": a / peak,
            "bytes": nbytes}


def flush_l2(buf):
    """Overwrite a buffer larger than L2 (between timed launches of small workloads)."""
    buf.add_(1.0)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--batch", type=int, default=B_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the ADMM, uneven-size and serving workloads")
    ap.add_argument("--extras", default="active30,branch256,admm,uneven,multiperiod,serving",
                    help="comma-separated subset of active30, branch256, admm, uneven, "
                         "multiperiod, serving")
    ap.add_argument("--admm-iters", type=int, default=1000)
    ap.add_argument("--mp-iters", type=int, default=200)
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--serve-cap-seconds", type=float, default=1.0 / 3.0,
                    help="the pool holds the buses, branches and generators offered in this "
                         "many seconds of arrivals (at least the largest instance)")
    ap.add_argument("--op-latency", action="store_true",
                    help="print the cycles per dependent FP64 / integer operation (1 and 32 "
                         "active lanes) as one JSON line instead of the benchmark")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="arrivals per second")
    ap.add_argument("--serve-sets", default="stated,convergent",
                    help="request sets to serve: stated, convergent")
    ap.add_argument("--serve-serial-prefix", type=int, default=0,
                    help="solve only the first N requests one at a time (FIFO latencies of a "
                         "prefix are exact); 0 = all")
    ap.add_argument("--serve-max-iters", type=int, default=200)
    ap.add_argument("--serve-conv-max-iters", type=int, default=6000)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (every 50 ms) of SM clock and throttle reasons."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([v.strip() for v in line.split(",")])

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------------- reference
def run_reference(args, rank, world):
    """The oracle (plain C, FP64) on this host's cores, same workload, sampled steps."""
    if rank != 0:
        return
    import oracle
    from paper_2106_14995_gb300 import synth
    cores = os.cpu_count() or 1
    sample = min(args.batch, 2000)
    d = synth.dense_batch(args.batch, N_VARS, seed_index=1)
    sub = {k: (v[:sample] if isinstance(v, np.ndarray) and v.ndim and v.shape[0] == args.batch
               else v) for k, v in d.items()}

    def step():
        return oracle.tron_batch(2, sub["params"], sub["l"], sub["u"], sub["x0"],
                                 sub["delta0"], nthreads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = step()
    dt = time.perf_counter() - t0
    assert (r["status"] == 0).all()
    value = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"dense quartic TRON, n=32, {args.batch} problems "
                               f"(first {sample} per step)", "global_batch": args.batch},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} of the {args.batch} problems per step, "
                                   f"{args.steps} steps, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- cpu baseline
def cpu_baseline(d, budget_s=12.0):
    """Oracle on the host cores over the whole batch, repeated for ~budget_s; also
    returns the oracle-counted algorithmic flops per problem on these inputs."""
    import oracle
    cores = os.cpu_count() or 1
    B = d["x0"].shape[0]
    t0 = time.perf_counter()
    reps, flops = 0, 0.0
    while True:
        r = oracle.tron_batch(2, d["params"], d["l"], d["u"], d["x0"], d["delta0"],
                              nthreads=cores)
        reps += 1
        flops = r["counters"]["flops"]
        if time.perf_counter() - t0 >= budget_s or reps >= 50:
            break
    dt = time.perf_counter() - t0
    # one thread, on the first 2,000 problems
    b1 = min(B, 2000)
    t1 = time.perf_counter()
    oracle.tron_batch(2, d["params"][:b1], d["l"][:b1], d["u"][:b1], d["x0"][:b1],
                      d["delta0"][:b1], nthreads=1)
    v1 = b1 / (time.perf_counter() - t1)
    return ({"value": B * reps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"the full {B}-problem batch solved {reps} time(s) on {cores} threads",
             "one_thread": {"value": v1, "unit": UNIT,
                            "sample": f"the first {b1} problems on 1 thread"}},
            flops / B, r)


# ---------------------------------------------------------------- extra workloads
def admm_bytes_per_iteration(nl, ng, nb):
    """Algorithmic HBM bytes of one component-ADMM iteration: per branch the record it
    reads (coefficients, multipliers, bus-side copies, warm start, limit) and the values
    it writes (352 B); per generator 96 B; per coupling pair the bus update's reads and
    writes of the two copies and the multiplier (40 B); 4 B per CSR incidence."""
    pairs = 8 * nl + 2 * ng
    return nl * 352 + ng * 96 + pairs * 40 + 4 * (2 * nl + ng + nb)


def bench_admm(args, dev, peak_measured):
    """Component ADMM on a 10,000-bus network (13,000 branches, 3,000 generators):
    ADMM iterations/s over args.admm_iters iterations (two launches per iteration, three
    when one-lane solves finish on four lanes; replayed CUDA graphs), with both branch
    mappings; the oracle runs the same
    iterations on the host cores (its time is the CPU baseline and its flop count the
    roofline's algorithmic work; the two trajectories agree to rounding)."""
    import torch
    import oracle
    from paper_2106_14995_gb300 import synth
    from paper_2106_14995_gb300.admm import Admm
    from paper_2106_14995_gb300.tron import options
    net = synth.network(10000, 3000, 3000, seed_index=2)
    nl, ng, nb = len(net["br_from"]), len(net["gen_bus"]), int(net["nbus"])

    def run(group, tr_norm=0, cauchy_norm=0):
        a = Admm(net, opts=options(group=group, tr_norm=tr_norm, cauchy_norm=cauchy_norm))
        grp = a.branch_group
        lpi = a.launches_per_iteration
        a.step(16)  # graph capture and the first iterations, untimed
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        pr, du = a.step(args.admm_iters)
        dt = time.perf_counter() - t0
        counts = a.branch_status_counts().tolist()
        a.close()
        return pr, du, dt, counts, grp, lpi

    # the library's mapping (chosen by the branch count), then the other one
    pr, du, dt, counts, grp, lpi = run(0)
    _, _, dt_o, _, grp_o, _ = run(4 if grp == 1 else 1)
    _, _, dt_e, _, _, _ = run(0, tr_norm=1)  # the other reading of the PCG's norm
    _, _, dt_h, _, _, _ = run(0, cauchy_norm=1)  # the Cauchy test in the Hessian's norm
    cores = os.cpu_count() or 1
    o = oracle.Admm(net)
    o.run(16, nthreads=cores)  # the iterations the GPU run did untimed
    f0 = o.counters.flops
    t1 = time.perf_counter()
    hp, hd = o.run(args.admm_iters, nthreads=cores)
    t_cpu = time.perf_counter() - t1
    flops_it = (o.counters.flops - f0) / args.admm_iters
    sec_it = dt / args.admm_iters
    return {"value": args.admm_iters / dt, "unit": "ADMM iters/s",
            "workload": "10,000 buses, 13,000 branches, 3,000 generators, rho=400",
            "iterations": args.admm_iters, "ms_per_iter": sec_it * 1e3,
            "gpu_launches": lpi * args.admm_iters, "final_primal": pr, "final_dual": du,
            "oracle_final": [float(hp[-1]), float(hd[-1])],
            "branch_status_last_iter": counts, "branch_lanes_per_problem": grp,
            "other_mapping": {"branch_lanes_per_problem": grp_o,
                              "value": args.admm_iters / dt_o, "unit": "ADMM iters/s"},
            "euclidean_reading": {"value": args.admm_iters / dt_e, "unit": "ADMM iters/s",
                                  "note": "options.tr_norm = 1 (PCG step bounded in ||w||_2)"},
            "hessian_cauchy": {"value": args.admm_iters / dt_h, "unit": "ADMM iters/s",
                               "note": "options.cauchy_norm = 1 (Cauchy test in (s'Hs)^(1/2))"},
            "roofline": fp64_roofline(flops_it, sec_it, peak_measured,
                                      f"k_admm_branch_gen<{grp}> + k_admm_bus",
                                      {"flops_per_iter": flops_it,
                                       "hbm": hbm_block(admm_bytes_per_iteration(nl, ng, nb),
                                                        sec_it)}),
            "cpu_baseline": {"value": args.admm_iters / t_cpu, "unit": "ADMM iters/s",
                             "cores": cores, "kind": "oracle",
                             "sample": f"the same {args.admm_iters} iterations (16 to "
                                       f"{16 + args.admm_iters})"}}


def bench_dense_active30(args, dev, peak_measured):
    """The headline family with c ~ N(0, 16^2) instead of N(0, 4^2): about 30 % of the
    bounds active at the solution (the share the workload description expects; the
    stated c gives 10 %), so more Cauchy breakpoints, newly active variables and
    multi-pass subspace loops.  10,000 problems, n = 32, autotuned persistent schedule,
    one launch at a time (median of five); roofline from the oracle's flop count on a
    2,000-problem sample."""
    import torch
    import oracle
    from paper_2106_14995_gb300 import native, synth
    from paper_2106_14995_gb300.tron import TronBatch, options
    d = synth.dense_batch(10000, N_VARS, seed_index=41, c_sd=16.0)
    B = 10000

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    P, L, U, X0, D0 = t(d["params"]), t(d["l"]), t(d["u"]), t(d["x0"]), t(d["delta0"])
    tb = TronBatch(2, B, n=N_VARS, opts=options(schedule=native.TRON_SCHED_PERSISTENT))
    tb.autotune(P, L, U, X0, D0, sample=4096)
    ts = []
    for rep in range(6):
        x, de = X0.clone(), D0.clone()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = tb.solve(P, L, U, x, de)
        e1.record()
        torch.cuda.synchronize(dev)
        if rep:
            ts.append(e0.elapsed_time(e1))
    xs = x.cpu().numpy()
    ok = bool((out["status"].cpu().numpy() == 0).all())
    tb.close()
    ms = float(np.median(ts))
    cores = os.cpu_count() or 1
    sub = {k: (v[:2000] if isinstance(v, np.ndarray) and v.ndim and v.shape[0] == B else v)
           for k, v in d.items()}
    r = oracle.tron_batch(2, sub["params"], sub["l"], sub["u"], sub["x0"], sub["delta0"],
                          nthreads=cores)
    flops = r["counters"]["flops"] / 2000 * B
    return {"value": B / (ms * 1e-3), "unit": UNIT, "ms": ms, "all_converged": ok,
            "active_bound_fraction": float(np.mean((xs <= d["l"]) | (xs >= d["u"]))),
            "workload": "10,000 dense quartic problems, n=32, c ~ N(0, 16^2)",
            "roofline": fp64_roofline(flops, ms * 1e-3, peak_measured,
                                      "k_tron_persistent<DenseObj<32,32>,32,32>",
                                      {"flops_per_launch": flops,
                                       "flops_from": "oracle, first 2,000 problems, scaled"})}


def bench_branch256(args, dev, peak_measured):
    """The 256 branch subproblems of one ADMM step (n = 4, cold start from the box
    midpoint, delta0 = 1): one batched solve per step, the library's mapping (four lanes
    per problem at this size) and the other one; L2 flushed between timed launches; end
    to end through the host-buffer path; the oracle on the host cores; roofline from the
    oracle's flop count.  A latency-bound configuration: 256 problems fill 32 warps."""
    import torch
    import oracle
    from paper_2106_14995_gb300 import synth
    from paper_2106_14995_gb300.tron import TronBatch, options
    d = synth.branch_batch(256, seed_index=0)
    B = 256

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    P, L, U, X0, D0 = t(d["params"]), t(d["l"]), t(d["u"]), t(d["x0"]), t(d["delta0"])
    scrub = torch.zeros(2 * L2_BYTES // 8, dtype=torch.float64, device=dev)
    res = {}
    for name, grp, trn, cn in (("default", 0, 0, 0), ("one_lane", 1, 0, 0),
                               ("four_lanes", 4, 0, 0), ("euclidean_reading", 0, 1, 0),
                               ("hessian_cauchy", 0, 0, 1)):
        tb = TronBatch(1, B, n=4, opts=options(group=grp, tr_norm=trn, cauchy_norm=cn))
        ts = []
        for rep in range(12):
            x, de = X0.clone(), D0.clone()
            flush_l2(scrub)
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = tb.solve(P, L, U, x, de)
            e1.record()
            torch.cuda.synchronize(dev)
            if rep >= 2:
                ts.append(e0.elapsed_time(e1))
        ok = bool((out["status"].cpu().numpy() == 0).all())
        res[name] = {"ms": float(np.median(ts)), "all_converged": ok,
                     "lanes_per_problem": int(tb.choices()[0]["group"]),
                     "max_iterations": int(out["iters"].max().item())}
        if name == "default":
            # end to end: pinned host inputs copied in, solved, results copied back
            hin = {k: torch.as_tensor(np.ascontiguousarray(d[k]), dtype=torch.float64)
                   .pin_memory() for k in ("params", "l", "u", "x0", "delta0")}
            tb.host_enable()
            hout = tb.host_outputs(B * 4)
            te = []
            for rep in range(12):
                t0 = time.perf_counter()
                tb.solve_host(hin["params"], hin["l"], hin["u"], hin["x0"], hin["delta0"], hout)
                tb.host_sync()
                if rep >= 2:
                    te.append(time.perf_counter() - t0)
            res["e2e_ms"] = float(np.median(te)) * 1e3
        tb.close()
    cores = os.cpu_count() or 1
    r = oracle.tron_batch(1, d["params"], d["l"], d["u"], d["x0"], d["delta0"], nthreads=cores)
    flops = r["counters"]["flops"]
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < 2.0:
        oracle.tron_batch(1, d["params"], d["l"], d["u"], d["x0"], d["delta0"], nthreads=cores)
        reps += 1
    cpu = B * reps / (time.perf_counter() - t0)
    ms = res["default"]["ms"]
    # algorithmic bytes: record 288 B, l, u, x0 96 B, delta 8 B in; x 32 B, delta, f,
    # pg 24 B, iterations and status 8 B out
    nbytes = B * (288 + 96 + 8 + 32 + 24 + 8)
    return {"value": B / (ms * 1e-3), "unit": UNIT, "ms": ms,
            "workload": "256 ACOPF branch subproblems (n=4), cold start, rho=400",
            "mappings": res, "e2e_ms": res["e2e_ms"],
            "roofline": fp64_roofline(flops, ms * 1e-3, peak_measured,
                                      "k_tron_plain<BranchObj<4>,4,4>",
                                      {"flops_per_launch": flops,
                                       "hbm": hbm_block(nbytes, ms * 1e-3),
                                       "note": "latency-bound: 256 problems fill 32 warps"}),
            "cpu_baseline": {"value": cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"the 256 problems solved {reps} times"}}


def bench_uneven(args, dev, peak_measured):
    """100,000 dense problems, n in {4,...,128} with probabilities (0.4, ..., 0.02):
    plain schedule (one launch per size class, in turn), persistent schedule (all
    classes concurrently, device work counters) and persistent after autotuning, and the
    last with the two other trust-region readings (options.tr_norm = 1, cauchy_norm = 1);
    the roofline's work is the oracle's flop count over the whole batch."""
    import torch
    import oracle
    from paper_2106_14995_gb300 import native, synth
    from paper_2106_14995_gb300.tron import TronBatch, options
    d = synth.uneven_batch(100000, seed_index=3)
    nv = d["nvec"]
    B = nv.size

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    P, L, U, X0, D0 = t(d["params"]), t(d["l"]), t(d["u"]), t(d["x0"]), t(d["delta0"])
    res = {}
    for name, sched, tune, extra in (
            ("plain", native.TRON_SCHED_PLAIN, False, {}),
            ("persistent", native.TRON_SCHED_PERSISTENT, False, {}),
            ("persistent_autotuned", native.TRON_SCHED_PERSISTENT, True, {}),
            ("euclidean_reading", native.TRON_SCHED_PERSISTENT, True, {"tr_norm": 1}),
            ("hessian_cauchy", native.TRON_SCHED_PERSISTENT, True, {"cauchy_norm": 1})):
        tb = TronBatch(2, B, n_list=nv, opts=options(schedule=sched, **extra))
        if tune:
            tb.autotune(P, L, U, X0, D0, sample=8192)
        ts = []
        for rep in range(6):  # the first untimed, then the median of five
            x, de = X0.clone(), D0.clone()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = tb.solve(P, L, U, x, de)
            e1.record()
            torch.cuda.synchronize(dev)
            if rep:
                ts.append(e0.elapsed_time(e1))
        ok = bool((out["status"].cpu().numpy() == 0).all())
        res[name] = {"value": B / (np.median(ts) * 1e-3), "unit": UNIT,
                     "ms": float(np.median(ts)), "launches": tb.last_launches,
                     "all_converged": ok}
        if extra:
            res[name]["note"] = ", ".join(f"options.{k} = {v}" for k, v in extra.items())
        # the kernel variant per size class (group/layout/warps per CTA) on stderr only
        print(f"uneven {name}: " + ", ".join(
            f"n={c['N']}:g{c['group']}/l{c['layout']}/w{c['warps_per_block']}"
            for c in tb.choices()), file=sys.stderr)
        tb.close()
    cores = os.cpu_count() or 1
    r = oracle.tron_batch(2, d["params"], d["l"], d["u"], d["x0"], d["delta0"], n=nv,
                          nthreads=cores)
    flops = r["counters"]["flops"]
    n64 = nv.astype(np.int64)
    nbytes = int(np.sum(8 * (n64 * n64 + 2 * n64) + 8 * 4 * n64 + 8 * 4 + 8))
    ms = res["persistent_autotuned"]["ms"]
    res["roofline"] = fp64_roofline(flops, ms * 1e-3, peak_measured,
                                    "k_tron_persistent (6 size classes, concurrent)",
                                    {"flops_per_launch": flops,
                                     "hbm": hbm_block(nbytes, ms * 1e-3)})
    res["workload"] = "100,000 dense problems, n in {4,6,8,16,32,64,128}"
    return res


def bench_multiperiod(args, dev, peak_measured):
    """Multi-period ADMM: 24 periods of a 2,000-bus network (2,600 branches, 600
    generators), loads on a synthetic daily profile, generators coupled by ramp limits of
    5 % of p_max (penalty 1e4): iterations/s over args.mp_iters iterations (five launches
    each: branches, the generator chains' gather, solve and scatter on a side stream
    beside them, buses; six with options.split_outer, which adds the branches' four-lane
    continuation); the oracle runs the same iterations on the host cores."""
    import torch
    import oracle
    from paper_2106_14995_gb300 import synth
    from paper_2106_14995_gb300.admm import AdmmMultiPeriod
    from paper_2106_14995_gb300.tron import options
    net = synth.network(2000, 600, 600, seed_index=9)
    T = 24
    scale = synth.load_profile(T)
    ramp = 0.05 * net["gen_pmax"]
    alt = {}
    for key, opt in (("euclidean_reading", options(tr_norm=1)),
                     ("hessian_cauchy", options(cauchy_norm=1)),
                     ("split_after_3", options(split_outer=3))):
        ge = AdmmMultiPeriod(net, scale, ramp=ramp, rho_ramp=1e4, opts=opt)
        ge.step(4)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ge.step(args.mp_iters)
        alt[key] = time.perf_counter() - t0
        ge.close()
    g = AdmmMultiPeriod(net, scale, ramp=ramp, rho_ramp=1e4)
    lpi = g.launches_per_iteration
    g.step(4)  # the first iterations, untimed
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    pr, du = g.step(args.mp_iters)
    dt = time.perf_counter() - t0
    counts = g.gen_status_counts().tolist()
    p = np.array([g.get_state(t)["gen_pq"][:, 0] for t in range(T)])
    g.close()
    cores = os.cpu_count() or 1
    o = oracle.MultiPeriodAdmm(net, scale, ramp=ramp, rho_ramp=1e4)
    o.run(4, nthreads=cores)
    f0 = o.counters.flops
    t1 = time.perf_counter()
    o.run(args.mp_iters, nthreads=cores)
    t_cpu = time.perf_counter() - t1
    nl, ng, nb = len(net["br_from"]), len(net["gen_bus"]), int(net["nbus"])
    sec_it = dt / args.mp_iters
    flops_it = (o.counters.flops - f0) / args.mp_iters
    return {"value": args.mp_iters / dt, "unit": "ADMM iters/s",
            "workload": "24 periods x (2,000 buses, 2,600 branches, 600 generators), "
                        "ramp 5 % of p_max, rho=400, rho_ramp=1e4",
            "iterations": args.mp_iters, "ms_per_iter": sec_it * 1e3,
            "gpu_launches": lpi * args.mp_iters, "final_primal": pr, "final_dual": du,
            "gen_status_last_iter": counts,
            "max_ramp_step_over_limit": float(np.max(np.abs(np.diff(p, axis=0)) -
                                                     ramp[None, :])),
            "euclidean_reading": {"value": args.mp_iters / alt["euclidean_reading"],
                                  "unit": "ADMM iters/s", "note": "options.tr_norm = 1"},
            "hessian_cauchy": {"value": args.mp_iters / alt["hessian_cauchy"],
                               "unit": "ADMM iters/s", "note": "options.cauchy_norm = 1"},
            "split_after_3": {"value": args.mp_iters / alt["split_after_3"],
                              "unit": "ADMM iters/s",
                              "note": "options.split_outer = 3: one-lane branch solves "
                                      "unfinished after 3 TRON iterations end on 4 lanes"},
            "roofline": fp64_roofline(flops_it, sec_it, peak_measured,
                                      "branch + generator-chain + bus kernels",
                                      {"flops_per_iter": flops_it,
                                       "hbm": hbm_block(T * admm_bytes_per_iteration(nl, ng, nb),
                                                        sec_it)}),
            "cpu_baseline": {"value": args.mp_iters / t_cpu, "unit": "ADMM iters/s",
                             "cores": cores, "kind": "oracle",
                             "sample": f"the same {args.mp_iters} iterations"}}


def _serve(reqs, tol, max_iters, chunk, cap_frac, serial_prefix=0):
    """Continuous batching of `reqs` in a pool that holds about cap_frac of their total
    buses, branches and generators (at least the largest instance), so arrivals wait for
    retirements; then the same requests one at a time (serial plain), or the first
    serial_prefix of them (a FIFO queue's latency of a request depends only on the
    requests before it, so the prefix's figures are exact; the served ones are then
    reported over the whole stream and over the same prefix)."""
    from paper_2106_14995_gb300.serving import AdmmServer, serial_plain, summarize
    tot = [sum(len(r["net"][k]) if k != "nbus" else r["net"][k] for r in reqs)
           for k in ("nbus", "br_from", "gen_bus")]
    big = [max(len(r["net"][k]) if k != "nbus" else r["net"][k] for r in reqs)
           for k in ("nbus", "br_from", "gen_bus")]
    cap = [max(int(cap_frac * t), b) + 128 * 8 for t, b in zip(tot, big)]
    n = len(reqs)
    srv = AdmmServer(cap[0], cap[1], cap[2], n, chunk=chunk, tol=tol, max_iters=max_iters)
    recs = srv.run(reqs)
    srv.close()
    waited = sum(1 for r in recs if r["admitted"] - r["arrival"] > 1e-3)
    served = summarize(recs)
    served["waited_for_admission"] = waited
    served["pool_capacity_buses"] = cap[0]
    served["offered_buses"] = tot[0]
    order = sorted(reqs, key=lambda q: q["t"])
    sreqs = order[:serial_prefix] if 0 < serial_prefix < len(order) else order
    serial = summarize(serial_plain(sreqs, chunk=chunk, tol=tol, max_iters=max_iters))
    out = {"served": served, "serial_plain": serial}
    ref = served
    if len(sreqs) < len(order):
        ids = {q["id"] for q in sreqs}
        ref = summarize([r for r in recs if r["id"] in ids])
        out["served_on_serial_prefix"] = ref
        out["serial_prefix"] = len(sreqs)
    out.update({"speedup_p50": serial["p50_s"] / ref["p50_s"],
                "speedup_p99": serial["p99_s"] / ref["p99_s"],
                "speedup_agg_iters": served["agg_iters_per_s"] / serial["agg_iters_per_s"]})
    return out


def bench_serving(args, dev):
    """Poisson arrivals (200/s over args.serve_seconds) of independent ADMM instances,
    served with continuous batching in a pool that holds the instances offered in
    args.serve_cap_seconds of arrivals (a third of a second by default), against the same
    requests solved one at a time (or the first args.serve_serial_prefix of them).

    * stated: bus counts log-uniform in [500, 20000] (branches 1.3x, generators 0.3x),
      load scaling U[0.8, 1.2], rho = 400, stop at both residuals <= 1e-4 or
      args.serve_max_iters iterations.  At these loads the networks cannot meet their
      loads inside the voltage box, so no instance reaches 1e-4: the times are to the cap.
    * convergent: the same arrival process with 500-2000 buses, a tenth of the load and
      rho = 10, stop at both residuals <= 1e-4 (cap args.serve_conv_max_iters): time to
      solution."""
    from paper_2106_14995_gb300 import synth
    out = {"unit": "s (time to solution)"}
    sets = set(args.serve_sets.split(","))
    rate, secs = args.serve_rate, args.serve_seconds
    cap_frac = min(1.0, args.serve_cap_seconds / secs)
    if "stated" in sets:
        specs = synth.serving_stream(duration_s=secs, rate_hz=rate)
        reqs = [dict(id=k, t=s["t"], net=synth.instance_network(s)) for k, s in enumerate(specs)]
        r = _serve(reqs, 1e-4, args.serve_max_iters, 10, cap_frac, args.serve_serial_prefix)
        r["workload"] = (f"{len(reqs)} instances over {secs} s at {rate:g}/s, buses "
                         f"log-U[500, 20000], load x U[0.8, 1.2], rho 400, stop at residuals "
                         f"<= 1e-4 or {args.serve_max_iters} iterations; pool for "
                         f"{args.serve_cap_seconds:.3g} s of arrivals")
        out["stated"] = r
    if "convergent" in sets:
        specs = synth.serving_stream(duration_s=secs, rate_hz=rate, seed_index=5,
                                     bus_lo=500, bus_hi=2000, load_lo=0.08, load_hi=0.12)
        reqs = [dict(id=k, t=s["t"], net=synth.instance_network(s), rho=10.0)
                for k, s in enumerate(specs)]
        r = _serve(reqs, 1e-4, args.serve_conv_max_iters, 20, cap_frac, args.serve_serial_prefix)
        r["workload"] = (f"{len(reqs)} instances over {secs} s at {rate:g}/s, buses "
                         f"log-U[500, 2000], load x U[0.08, 0.12], rho 10, stop at residuals "
                         f"<= 1e-4 (cap {args.serve_conv_max_iters}); pool for "
                         f"{args.serve_cap_seconds:.3g} s of arrivals")
        out["convergent"] = r
    return out


def finite_or_null(v):
    """The JSON line with non-finite numbers (percentiles of empty sets) as null."""
    if isinstance(v, float):
        return v if np.isfinite(v) else None
    if isinstance(v, dict):
        return {k: finite_or_null(x) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [finite_or_null(x) for x in v]
    return v


def summary(line: dict) -> dict:
    """The key figure of every workload in a few hundred characters (placed last in the
    JSON line, so that a reader of the output's tail sees all of them)."""
    def r(v, k=4):
        return None if v is None else float(f"{v:.{k}g}")
    out = {"dense32": {"subproblems_per_s": r(line["value"]),
                       "e2e": r(line["e2e"]["value"])}}
    rf = line.get("roofline")
    if rf:
        out["dense32"].update(frac=r(rf["frac"], 3), frac_measured=r(rf.get("frac_measured"), 3),
                              fp64_peak_measured=r(rf.get("peak_measured")),
                              cpu=r(line["cpu_baseline"]["value"]))
    a30 = line.get("dense_active30")
    if a30:
        out["dense32_active30"] = {"subproblems_per_s": r(a30["value"]),
                                   "active": r(a30["active_bound_fraction"], 3),
                                   "frac": r(a30["roofline"]["frac"], 3)}
    b = line.get("branch256")
    if b:
        out["branch256"] = {"ms": r(b["ms"]), "subproblems_per_s": r(b["value"]),
                            "e2e_ms": r(b["e2e_ms"]),
                            "euclidean_ms": r(b["mappings"]["euclidean_reading"]["ms"]),
                            "hessian_cauchy_ms": r(b["mappings"]["hessian_cauchy"]["ms"]),
                            "cpu": r(b["cpu_baseline"]["value"])}
    a = line.get("admm")
    if a:
        out["admm10k"] = {"iters_per_s": r(a["value"]), "frac": r(a["roofline"]["frac"], 3),
                          "other_mapping": r(a["other_mapping"]["value"]),
                          "euclidean": r(a["euclidean_reading"]["value"]),
                          "hessian_cauchy": r(a["hessian_cauchy"]["value"]),
                          "cpu": r(a["cpu_baseline"]["value"])}
    u = line.get("uneven")
    if u:
        out["uneven100k_ms"] = {"plain": r(u["plain"]["ms"]),
                                "persistent": r(u["persistent"]["ms"]),
                                "autotuned": r(u["persistent_autotuned"]["ms"]),
                                "euclidean": r(u["euclidean_reading"]["ms"]),
                                "hessian_cauchy": r(u["hessian_cauchy"]["ms"]),
                                "frac": r(u["roofline"]["frac"], 3),
                                "frac_measured": r(u["roofline"].get("frac_measured"), 3)}
    m = line.get("multiperiod")
    if m:
        out["multiperiod"] = {"iters_per_s": r(m["value"]),
                              "euclidean": r(m["euclidean_reading"]["value"]),
                              "hessian_cauchy": r(m["hessian_cauchy"]["value"]),
                              "split_after_3": r(m["split_after_3"]["value"]),
                              "cpu": r(m["cpu_baseline"]["value"])}
    sv = line.get("serving")
    if sv:
        for k in ("stated", "convergent"):
            if k not in sv:
                continue
            x = sv[k]
            out["serving_" + k] = {
                "n": x["served"]["instances"], "converged": x["served"]["converged"],
                "waited": x["served"]["waited_for_admission"],
                "p50_s": r(x["served"]["p50_s"], 3), "p99_s": r(x["served"]["p99_s"], 3),
                "serial_p50_s": r(x["serial_plain"]["p50_s"], 3),
                "serial_p99_s": r(x["serial_plain"]["p99_s"], 3),
                "p50_converged_s": r(x["served"]["p50_converged_s"], 3),
                "serial_p50_converged_s": r(x["serial_plain"]["p50_converged_s"], 3),
                "iters_per_s": r(x["served"]["agg_iters_per_s"]),
                "serial_iters_per_s": r(x["serial_plain"]["agg_iters_per_s"])}
    return out


# -------------------------------------------------------------------- main arm
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    if args.op_latency:
        from paper_2106_14995_gb300.tron import OP_LATENCY_NAMES, op_latency
        table = {name: {"lanes_1": round(op_latency(k, 1), 1), "lanes_32": round(op_latency(k, 32), 1)}
                 for k, name in enumerate(OP_LATENCY_NAMES)}
        print(json.dumps({"metric": "SM cycles per dependent operation (chain of 2048, one CTA)",
                          "ops": table}))
        return 0

    import torch
    import torch.distributed as dist
    from paper_2106_14995_gb300 import _build, native, synth
    from paper_2106_14995_gb300 import dist as xdist
    from paper_2106_14995_gb300.tron import TronBatch, options

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:  # one rank compiles (if anything is stale); the others wait for it
        _build.build()
    if world > 1:
        dist.barrier()
    native.load()

    # weak scaling: every rank solves its own batch of the same distribution (rank 0
    # the canonical seeded batch, rank r > 0 an independent draw); no data-path
    # collective, only the timing is combined
    if rank == 0:
        d = synth.dense_batch(args.batch, N_VARS, seed_index=1)
    else:
        rng = synth.rng_for(1, salt=rank)
        rec, lo_, hi_, x0_ = synth.dense_records(rng, args.batch, N_VARS)
        d = dict(kind=2, n=N_VARS, params=rec, l=lo_, u=hi_, x0=x0_,
                 delta0=np.ones(args.batch))
    B = args.batch
    stream = torch.cuda.Stream(device=dev)

    def t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)

    params, lo, hi = t(d["params"]), t(d["l"]), t(d["u"])
    x0, d0 = t(d["x0"]), t(d["delta0"])
    bytes_in = (params.numel() + lo.numel() + hi.numel() + x0.numel() + d0.numel()) * 8
    nbuf = max(2, int(np.ceil(2 * L2_BYTES / bytes_in)) + 1)
    bufs = [dict(p=params.clone(), l=lo.clone(), u=hi.clone()) for _ in range(nbuf)]
    # a fresh x0 and delta0 for every step: warm-up, the timed steps and the serial
    # per-launch timing after them
    nsteps = args.warmup + 2 * args.steps
    xs = [x0.clone() for _ in range(nsteps)]
    ds = [d0.clone() for _ in range(nsteps)]

    def outputs():
        return dict(f=torch.empty(B, dtype=torch.float64, device=dev),
                    pg=torch.empty(B, dtype=torch.float64, device=dev),
                    iters=torch.empty(B, dtype=torch.int32, device=dev),
                    status=torch.empty(B, dtype=torch.int32, device=dev))
    # consecutive steps alternate between two streams, each with its own outputs: a
    # step's last wave overlaps the next step's start (the handle gives concurrent
    # solves their own work counters)
    streams = [stream, torch.cuda.Stream(device=dev)]
    outs = [outputs(), outputs()]
    # the library's tuned path: autotune once at setup (outside the timed region) on a
    # sample of this batch, then the persistent schedule
    tb = TronBatch(2, B, n=N_VARS, opts=options(schedule=native.TRON_SCHED_PERSISTENT),
                   stream=stream)
    tuned = tb.autotune(params, lo, hi, x0, d0, sample=min(B, 4096), stream=stream)

    def step(i, si):
        b = bufs[i % nbuf]
        tb.solve(b["p"], b["l"], b["u"], xs[i], ds[i], stream=streams[si], **outs[si])

    for i in range(args.warmup):
        step(i, i % 2)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    s1_done = torch.cuda.Event()
    launches = 0
    t_start.record(streams[0])
    streams[1].wait_event(t_start)
    for k in range(args.steps):
        step(args.warmup + k, k % 2)
        launches += tb.last_launches
    s1_done.record(streams[1])
    streams[0].wait_event(s1_done)
    t_end.record(streams[0])
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    used = outs if args.steps > 1 else outs[:1]  # a single step writes one output set
    ok = all(bool((o["status"].cpu().numpy() == 0).all() and
                  (o["pg"].cpu().numpy() <= 1e-6).all()) for o in used)
    # the kernel alone: the same number of launches one after another on one stream,
    # each bracketed by events (the roofline's per-launch duration)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        ev[k][0].record(streams[0])
        step(args.warmup + args.steps + k, 0)
        ev[k][1].record(streams[0])
    torch.cuda.synchronize(dev)
    launch_ms = [a.elapsed_time(b) for a, b in ev]
    ok = ok and bool((outs[0]["status"].cpu().numpy() == 0).all())
    # share of the variables at a bound in the last solution
    xa = xs[-1].cpu().numpy()
    active = float(np.mean((xa <= d["l"]) | (xa >= d["u"])))
    total_ms = xdist.max_over_ranks(total_ms, device=dev)
    value = xdist.weak_scaling_throughput(B, world, args.steps, total_ms)

    # end to end through the C ABI's host-buffer path (tron_batch_solve_host): every step
    # copies its inputs from pinned host memory to the device and its results (x, delta,
    # f, pg, iters, status) back; consecutive steps overlap through the library's two
    # device buffer sets.  Wall clock from the first call to the last result in host memory.
    host_in = {k: torch.as_tensor(np.ascontiguousarray(d[k]), dtype=torch.float64).pin_memory()
               for k in ("params", "l", "u", "x0", "delta0")}
    tb.host_enable()
    hout = [tb.host_outputs(B * N_VARS) for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = sum(v.numel() * v.element_size() for v in hout[0].values())

    def e2e_step(i):
        tb.solve_host(host_in["params"], host_in["l"], host_in["u"], host_in["x0"],
                      host_in["delta0"], hout[i % 2])

    for i in range(args.warmup):
        e2e_step(i)
    tb.host_sync()
    if world > 1:
        dist.barrier()
    e0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    tb.host_sync()
    e2e_ms = (time.perf_counter() - e0) * 1e3
    e2e_ok = all(bool((h["status"].numpy() == 0).all()) for h in hout)
    ok = ok and e2e_ok
    e2e_ms = xdist.max_over_ranks(e2e_ms, device=dev)
    e2e_value = xdist.weak_scaling_throughput(B, world, args.steps, e2e_ms)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded; stands in for the paper's branch batches)",
        "config": {"workload": f"batched TRON, dense quartic, n={N_VARS}, {B} problems per GPU",
                   "global_batch": world * B, "n": N_VARS, "gtol": 1e-6,
                   "schedule": "persistent",
                   "kernel_choice": ", ".join(f"n={c['N']}:g{c['group']}/l{c['layout']}/"
                                              f"w{c['warps_per_block']}" for c in tuned),
                   "parallelism": f"replicas x{world} (independent problems per GPU)",
                   "l2": f"inputs larger than L2: {nbuf} rotating copies of the batch",
                   "overlap": "consecutive steps alternate between two streams (one step's "
                              "last wave overlaps the next one's start); roofline launch "
                              "times are taken with launches one at a time"},
        "all_converged": ok,
        "active_bound_fraction": active,
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "path": "tron_batch_solve_host (pinned host buffers)"},
    }
    peak_measured = fp64_peak_measured(dev, native.load()) if rank == 0 else None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, flops_per_problem, _ = cpu_baseline(d)
        achieved = flops_per_problem * B / (float(np.median(launch_ms)) * 1e-3) / 1e9
        lms = float(np.median(launch_ms))
        ex = executed_flops_per_launch(B)
        line["roofline"] = {
            "bound": "alu", "kernel": "k_tron_persistent<DenseObj<32,32>,32,32>",
            "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
            "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic_per_launch(B),
            "flops_per_launch": flops_per_problem * B,
            "executed_flops_per_launch": ex,
            "executed_frac": (ex / (lms * 1e-3) / 1e9 / FP64_PEAK_GFLOPS) if ex else None,
            "launch_ms_median": lms,
            # the timed region's launches back to back (one step's last wave overlapping
            # the next one's start): the time each adds, not a launch's own duration
            "overlapped": {"ms_per_launch": total_ms / args.steps,
                           "achieved": flops_per_problem * B / (total_ms / args.steps * 1e-3)
                           / 1e9,
                           "frac": flops_per_problem * B / (total_ms / args.steps * 1e-3)
                           / 1e9 / FP64_PEAK_GFLOPS},
            "hbm": {"achieved": ALG_BYTES_PER_PROBLEM * B / (lms * 1e-3) / 1e9,
                    "peak": hbm_peak_gbs()[0], "peak_source": hbm_peak_gbs()[1],
                    "unit": "GB/s",
                    "frac": ALG_BYTES_PER_PROBLEM * B / (lms * 1e-3) / 1e9 / hbm_peak_gbs()[0]},
            "peak_measured": peak_measured,
            "frac_measured": (achieved / peak_measured) if peak_measured else None,
            "note": "FP64 CUDA-core pipe; peak from 2 DFMA/clk/SM x 152 SMs x 2.07 GHz, "
                    "peak_measured from the library's FP64 FMA probe in this run; "
                    "achieved counts the oracle's algorithmic flops, executed_frac the "
                    "FP64 flops the kernel issues (ncu thread-level counts)"}
        line["cpu_baseline"] = cb
    tb.close()
    if rank == 0 and world == 1 and not args.no_extras:
        extras = set(args.extras.split(","))
        if "active30" in extras:
            line["dense_active30"] = bench_dense_active30(args, dev, peak_measured)
        if "branch256" in extras:
            line["branch256"] = bench_branch256(args, dev, peak_measured)
        if "admm" in extras:
            line["admm"] = bench_admm(args, dev, peak_measured)
        if "uneven" in extras:
            line["uneven"] = bench_uneven(args, dev, peak_measured)
        if "multiperiod" in extras:
            line["multiperiod"] = bench_multiperiod(args, dev, peak_measured)
        if "serving" in extras:
            line["serving"] = bench_serving(args, dev)
    if rank == 0:
        line["summary"] = summary(line)
    if rank == 0:
        print(json.dumps(finite_or_null(line), allow_nan=False), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
