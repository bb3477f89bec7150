"""The serving loop's host logic on CPU, against a stand-in pool: admission by capacity
in arrival order (first come, first served), retirement at the residual tolerance or the
iteration cap, slots reused, and the latency summary.  The stand-in keeps each
instance's iteration count and lets its residuals fall geometrically; time is a fake
clock that the pool's steps (and every look at the clock) advance."""
import numpy as np
import pytest

from paper_2106_14995_gb300.serving import AdmmServer, summarize


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1e-4  # every look at the clock takes a little time
        return self.t


class FakePool:
    """Capacity in buses; instance k's residuals after i iterations: r0_k * decay_k^i."""

    def __init__(self, cap_bus, clock, step_s=1e-3):
        self.cap = cap_bus
        self.clock = clock
        self.step_s = step_s
        self.live = {}
        self.next_id = 0
        self.max_live = 0
        self.admitted_order = []

    def add(self, net):
        used = sum(v["nbus"] for v in self.live.values())
        if used + net["nbus"] > self.cap:
            return None
        i = self.next_id
        self.next_id += 1
        self.live[i] = dict(nbus=net["nbus"], it=0, r0=net["r0"], decay=net["decay"],
                            name=net["name"])
        self.admitted_order.append(net["name"])
        self.max_live = max(self.max_live, len(self.live))
        return i

    def step(self, n):
        for v in self.live.values():
            v["it"] += n
        self.clock.t += self.step_s

    def residuals(self):
        m = self.next_id
        it = np.zeros(m, dtype=np.int64)
        pr = np.full(m, np.inf)
        du = np.full(m, np.inf)
        for i, v in self.live.items():
            it[i] = v["it"]
            pr[i] = du[i] = v["r0"] * v["decay"] ** v["it"]
        return it, pr, du

    def remove(self, i):
        del self.live[i]

    def get_state(self, i):
        return dict(iteration=self.live[i]["it"])

    def close(self):
        pass


def _req(name, t, nbus, decay, r0=1.0):
    return dict(id=name, t=t, net=dict(nbus=nbus, r0=r0, decay=decay, name=name))


def test_admission_by_capacity_and_retirement():
    clock = FakeClock()
    pool = FakePool(cap_bus=200, clock=clock)
    srv = AdmmServer(0, 0, 0, 0, chunk=4, tol=1e-3, max_iters=400, pool=pool)
    reqs = [_req("a", 0.0, 100, 0.5), _req("b", 0.0, 100, 0.9), _req("c", 0.0, 100, 0.5),
            _req("d", 0.0005, 50, 1.0)]  # d never converges: retired at the cap
    out = {r["id"]: r for r in srv.run(reqs, clock=clock, keep_state=True)}
    assert set(out) == {"a", "b", "c", "d"}
    assert pool.max_live <= 2                      # 200 buses hold two 100-bus instances
    # first come, first served: c waits for a slot although d would fit beside a and b
    assert pool.admitted_order == ["a", "b", "c", "d"]
    # a: 0.5^i <= 1e-3 from i = 10, seen at the next chunk boundary (12)
    assert out["a"]["converged"] and out["a"]["iterations"] == 12
    assert out["b"]["converged"] and out["b"]["iterations"] == 68   # 0.9^i <= 1e-3: i >= 66
    assert not out["d"]["converged"] and out["d"]["iterations"] == 400
    assert out["a"]["state"]["iteration"] == 12
    for r in out.values():
        assert r["arrival"] <= r["admitted"] <= r["finished"]
    assert out["c"]["admitted"] >= out["a"]["finished"]    # into a's freed slots
    assert not pool.live


def test_arrivals_in_the_future_are_waited_for():
    clock = FakeClock()
    pool = FakePool(cap_bus=1000, clock=clock)
    srv = AdmmServer(0, 0, 0, 0, chunk=8, tol=1e-2, max_iters=1000, pool=pool)
    reqs = [_req("late", 0.05, 10, 0.5), _req("early", 0.0, 10, 0.5)]
    out = {r["id"]: r for r in srv.run(reqs, clock=clock)}
    assert pool.admitted_order == ["early", "late"]
    assert out["late"]["admitted"] >= 0.05
    assert out["early"]["iterations"] == out["late"]["iterations"] == 8


def test_summary_percentiles_and_throughput():
    recs = [dict(arrival=0.0, finished=1.0, iterations=100, converged=True),
            dict(arrival=0.5, finished=2.5, iterations=300, converged=False),
            dict(arrival=1.0, finished=4.0, iterations=200, converged=True)]
    s = summarize(recs)
    assert s["instances"] == 3 and s["iterations"] == 600 and s["converged"] == 2
    assert s["p50_s"] == pytest.approx(2.0)
    assert s["p99_s"] == pytest.approx(np.percentile([1.0, 2.0, 3.0], 99))
    assert s["makespan_s"] == pytest.approx(4.0)
    assert s["agg_iters_per_s"] == pytest.approx(150.0)
