"""bench.py's output contract where it needs no GPU: the reference arm (the oracle timed
on the host cores) prints one JSON line with the keys the harness reads; the CPU
baseline and the HBM peak lookup behave as documented."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["unit"] == "subproblems/s"
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert "workload" in line["config"]


def test_cpu_baseline_and_peak_lookup():
    import bench
    from paper_2106_14995_gb300 import synth
    d = synth.dense_batch(64, bench.N_VARS, seed_index=1)
    cb, flops, r = bench.cpu_baseline(d, budget_s=0.0)
    assert cb["value"] > 0 and cb["cores"] >= 1 and cb["kind"] == "oracle"
    assert cb["one_thread"]["value"] > 0
    assert flops > 0 and (r["status"] == 0).all()
    peak, src = bench.hbm_peak_gbs()
    assert peak > 0 and src in ("measured", "fallback")
    # the algorithmic bytes of one n = 32 problem: record, bounds, x0, delta in; x,
    # delta, f, pg, iterations, status out
    assert bench.ALG_BYTES_PER_PROBLEM == 8 * (32 * 32 + 64) + 3 * 256 + 8 + 256 + 24 + 8
