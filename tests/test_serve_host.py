"""Host logic of the continuous-batching scheduler (no GPU): admission by HBM budget and slots,
arrival order, rounds, retirement, failure isolation and latency accounting, driven by a fake
engine and a deterministic clock."""
import numpy as np

from paper_0801_4169_gb300 import serve
from paper_0801_4169_gb300 import workloads as W


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeEngine:
    """Each step of each active solve costs 1 ms of fake time; requests with Ms > 9 'fail'."""

    def __init__(self, clock):
        self.clock = clock
        self.steps = {}
        self.live = set()
        self.peak_live = 0

    def nbytes(self, req):
        return req.nx * 1000

    def create(self, req):
        s = object()
        self.steps[s] = (req, 0)
        self.live.add(s)
        self.peak_live = max(self.peak_live, len(self.live))
        return s

    def step(self, solves, k):
        self.clock.t += 1e-3 * k * len(solves)
        failed = {}
        for s in solves:
            req, n = self.steps[s]
            self.steps[s] = (req, n + k)
            if req.Ms > 9.0:
                failed[s] = "numeric"
        return failed

    def result(self, s):
        return self.steps[s][1]

    def release(self, s):
        self.live.discard(s)

    def close(self):
        pass


def _reqs(n=40, seed=3):
    rs = W.serving_requests(n=n, seed=seed, nx_range=(256, 2048), steps_range=(100, 1000))
    return rs


def test_every_request_finishes_with_its_own_step_count():
    clk = FakeClock()
    eng = FakeEngine(clk)
    sch = serve.Scheduler(eng, budget_bytes=10 ** 9, round_steps=50, clock=clk)
    reqs = _reqs()
    out = sch.run(reqs, realtime=False)
    done = [j for j in sch.finished if j.status == "done"]
    failed = [j for j in sch.finished if j.status == "failed"]
    assert len(done) + len(failed) == len(reqs)
    for j in done:
        assert j.result == j.req.steps  # never over- or under-stepped
        assert j.finished_s >= j.req.arrival_s
    assert all(j.req.Ms > 9.0 for j in failed) and len(failed) == sum(r.Ms > 9.0 for r in reqs)
    assert out["requests_done"] == len(done) and out["p99_s"] >= out["p50_s"]


def test_budget_and_slots_bound_admission():
    clk = FakeClock()
    eng = FakeEngine(clk)
    budget = 4 * 2048 * 1000
    sch = serve.Scheduler(eng, budget_bytes=budget, max_slots=3, round_steps=50, clock=clk)
    sch.run(_reqs(), realtime=False)
    assert sch.stats.max_bytes <= budget
    assert sch.stats.max_active <= 3 and eng.peak_live <= 3


def test_admission_is_in_arrival_order():
    clk = FakeClock()
    eng = FakeEngine(clk)
    sch = serve.Scheduler(eng, budget_bytes=10 ** 9, max_slots=2, round_steps=50, clock=clk)
    reqs = _reqs(n=12)
    sch.run(reqs, realtime=False)
    adm = sorted((j.admitted_s, j.req.arrival_s) for j in sch.finished if j.admitted_s is not None)
    arrivals = [a for _, a in adm]
    assert arrivals == sorted(arrivals)


def test_failed_request_does_not_stop_the_others():
    clk = FakeClock()
    eng = FakeEngine(clk)
    sch = serve.Scheduler(eng, budget_bytes=10 ** 9, round_steps=50, clock=clk)
    reqs = _reqs(n=20, seed=5)
    bad = sum(r.Ms > 9.0 for r in reqs)
    assert 0 < bad < len(reqs)
    sch.run(reqs, realtime=False)
    assert sch.stats.failed == bad
    assert len([j for j in sch.finished if j.status == "done"]) == len(reqs) - bad


def test_oversized_request_is_refused():
    clk = FakeClock()
    eng = FakeEngine(clk)
    sch = serve.Scheduler(eng, budget_bytes=1000, round_steps=50, clock=clk)
    job = sch.submit(_reqs(n=1)[0])
    assert job.status == "failed" and "budget" in job.error


def test_latency_includes_queueing():
    """With one slot, the second request's time to solution includes waiting for the first."""
    clk = FakeClock()
    eng = FakeEngine(clk)
    sch = serve.Scheduler(eng, budget_bytes=10 ** 9, max_slots=1, round_steps=1000, clock=clk)
    r1 = W.Request(0, 0.0, 512, 4, 3.0, 100, 0)
    r2 = W.Request(1, 0.0, 512, 4, 3.0, 100, 0)
    sch.run([r1, r2], realtime=False)
    lat = sorted(sch.stats.latencies)
    assert np.isclose(lat[0], 0.1) and np.isclose(lat[1], 0.2)
