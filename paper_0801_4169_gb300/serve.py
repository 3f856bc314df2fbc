"""Continuous-batching server for FDLBM solves on one GPU.

Requests (a shock-tube solve: grid, Mach number, step count, storage precision) arrive over
time. Each round the server does the following:

1. Admit queued requests in arrival order, while the HBM budget and the slot count allow.
2. Advance every admitted solve by the same number of steps. Each precision group is one
   batch: one kernel launch per time step over all of its members (fdlbm_batch_step).
3. Retire finished solves (moments read back) and failed ones (a sticky numerical error is
   reported, never silently upgraded to FP64).
4. Record each request's time to solution (finish time minus arrival time).

Requests that arrive while others are on the GPU join at the next round, as memory and slots
free up. Their device work then overlaps with everyone else's inside the same launches.

The scheduler (Scheduler) is engine-agnostic host logic. GpuEngine runs it on the library, and
tests drive it with a fake engine. mode="separate" is the baseline: one launch sequence per
solve (fdlbm_step on each handle), no packing.

    python -m paper_0801_4169_gb300.serve --requests 512 [--mode batched|separate] [--prec mixed|fp64]
"""
import argparse
import json
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as W


@dataclass
class Job:
    req: W.Request
    nbytes: int = 0
    solve: object = None
    done: int = 0
    admitted_s: float = None
    finished_s: float = None
    status: str = "queued"    # queued, active, done, failed
    result: tuple = None
    error: str = ""

    @property
    def remaining(self):
        return self.req.steps - self.done


@dataclass
class Stats:
    latencies: list = field(default_factory=list)
    lups: float = 0.0
    wall_s: float = 0.0
    rounds: int = 0
    max_active: int = 0
    max_bytes: int = 0
    failed: int = 0

    def summary(self):
        lat = np.array(self.latencies) if self.latencies else np.array([np.nan])
        return {"requests_done": len(self.latencies), "failed": self.failed,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "mean_s": float(np.mean(lat)), "aggregate_glups": self.lups / max(self.wall_s, 1e-12) / 1e9,
                "wall_s": self.wall_s, "rounds": self.rounds, "max_active": self.max_active,
                "max_bytes": self.max_bytes}


class Scheduler:
    """Admission by HBM budget and slots, rounds of `round_steps`, retirement, latency accounting."""

    def __init__(self, engine, budget_bytes=1 << 30, max_slots=256, round_steps=500, clock=None):
        self.engine = engine
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.round_steps = int(round_steps)
        self.clock = clock or time.perf_counter
        self.queue = []
        self.active = []
        self.finished = []
        self.stats = Stats()
        self.used = 0

    def submit(self, req):
        job = Job(req=req, nbytes=self.engine.nbytes(req))
        if job.nbytes > self.budget:
            job.status = "failed"
            job.error = "larger than the HBM budget"
            self.finished.append(job)
            self.stats.failed += 1
            return job
        self.queue.append(job)
        return job

    def _admit(self, now):
        while self.queue and len(self.active) < self.max_slots:
            job = self.queue[0]
            if self.used + job.nbytes > self.budget:
                break  # arrival order: the head of the queue waits for memory
            self.queue.pop(0)
            job.solve = self.engine.create(job.req)
            job.admitted_s = now
            job.status = "active"
            self.active.append(job)
            self.used += job.nbytes
        self.stats.max_active = max(self.stats.max_active, len(self.active))
        self.stats.max_bytes = max(self.stats.max_bytes, self.used)

    def _retire(self, job, now, failed=False, error=""):
        self.active.remove(job)
        self.used -= job.nbytes
        job.finished_s = now
        if failed:
            job.status = "failed"
            job.error = error
            self.stats.failed += 1
        else:
            job.status = "done"
            job.result = self.engine.result(job.solve)
            self.stats.latencies.append(now - job.req.arrival_s)
        self.engine.release(job.solve)
        job.solve = None
        self.finished.append(job)

    def round(self, now):
        """Admit, advance all active solves by k steps, retire. Returns the steps taken (0 if idle)."""
        self._admit(now)
        if not self.active:
            return 0
        k = min(self.round_steps, min(j.remaining for j in self.active))
        failed = self.engine.step([j.solve for j in self.active], k)
        for j in self.active:
            j.done += k
        self.stats.lups += k * sum(j.req.nx * j.req.ny for j in self.active)
        self.stats.rounds += 1
        t = self.clock() - self._t0
        for j in list(self.active):
            if j.solve in failed:
                self._retire(j, t, failed=True, error=failed[j.solve])
            elif j.remaining == 0:
                self._retire(j, t)
        return k

    def run(self, requests, realtime=True):
        """Serve a stream. realtime=True replays arrival times on the wall clock; False admits a
        request as soon as the clock has passed its arrival, without sleeping (virtual time)."""
        pending = sorted(requests, key=lambda r: r.arrival_s)
        self._t0 = self.clock()
        i = 0
        while i < len(pending) or self.queue or self.active:
            now = self.clock() - self._t0
            if not realtime:
                # virtual time: everything that would have arrived by now, else jump to the next arrival
                if not self.active and not self.queue and i < len(pending):
                    self._t0 -= max(0.0, pending[i].arrival_s - now)
                    now = self.clock() - self._t0
            while i < len(pending) and pending[i].arrival_s <= now:
                self.submit(pending[i])
                i += 1
            if self.round(now) == 0 and i < len(pending):
                if realtime:
                    time.sleep(max(0.0, min(0.01, pending[i].arrival_s - (self.clock() - self._t0))))
        self.stats.wall_s = self.clock() - self._t0
        self.engine.close()
        return self.stats.summary()


class GpuEngine:
    """Runs solves on the CUDA library: one batch per (precision) group, or separate launches."""

    def __init__(self, mode="batched", lam=2.0, force_prec=None, autotune=False):
        import torch
        from . import fdlbm as F
        self.F = F
        self.torch = torch
        self.mode = mode
        self.lam = lam
        self.force_prec = force_prec
        self.autotune = autotune
        self.stream = torch.cuda.Stream()
        self.batches = {}

    def _prec(self, req):
        return req.prec if self.force_prec is None else self.force_prec

    def nbytes(self, req):
        F = self.F
        w = W.request_workload(req, lam=self.lam)
        cfg = F.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, self._prec(req))
        return F.fdlbm_device_bytes(cfg)

    def create(self, req):
        F = self.F
        w = W.request_workload(req, lam=self.lam)
        s = F.Solver(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, self._prec(req), 0, w.bstate,
                     stream=self.stream)
        s.set_macro(*w.macros())
        s.prec = self._prec(req)
        if self.mode == "batched":
            b = self.batches.get(s.prec)
            if b is None:
                b = self.batches[s.prec] = F.fdlbm_batch_create(self.stream)
            F.fdlbm_batch_add(b, s.h)
            s.batch = b
        return s

    def step(self, solves, k):
        """Advance all solves k steps; returns {solve: error message} for those that failed."""
        F = self.F
        failed = {}
        if self.mode == "batched":
            for prec, b in self.batches.items():
                if F.fdlbm_batch_size(b) == 0:
                    continue
                if self.autotune and getattr(self, "_tuned_%d" % prec, 0) != F.fdlbm_batch_size(b):
                    F.fdlbm_batch_autotune(b, 2)
                    setattr(self, "_tuned_%d" % prec, F.fdlbm_batch_size(b))
                F.fdlbm_batch_step(b, k)
            any_failed = 0
            for prec, b in self.batches.items():
                if F.fdlbm_batch_size(b):
                    any_failed += F.fdlbm_batch_sync(b)[0]
            if any_failed:  # rare: find the members carrying the sticky error
                for s in solves:
                    try:
                        F.fdlbm_sync(s.h)
                    except F.FdlbmError as e:
                        failed[s] = str(e)
        else:
            for s in solves:
                F.fdlbm_step(s.h, k)
            for s in solves:
                try:
                    F.fdlbm_sync(s.h)
                except F.FdlbmError as e:
                    failed[s] = str(e)
        return failed

    def result(self, s):
        return s.get_macro(check=False)

    def release(self, s):
        F = self.F
        b = getattr(s, "batch", None)
        if b is not None:
            F.fdlbm_batch_remove(b, s.h)
            s.batch = None
        s.close()

    def close(self):
        for b in self.batches.values():
            self.F.fdlbm_batch_destroy(b)
        self.batches = {}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--mode", default="batched", choices=["batched", "separate"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--budget-gib", type=float, default=1.0)
    ap.add_argument("--round-steps", type=int, default=500)
    ap.add_argument("--steps-scale", type=float, default=1.0, help="scale every request's step count")
    ap.add_argument("--virtual", action="store_true", help="virtual arrival clock (no sleeping)")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    reqs = W.serving_requests(n=args.requests, seed=args.seed)
    for r in reqs:
        r.steps = max(1, int(round(r.steps * args.steps_scale)))
    eng = GpuEngine(mode=args.mode, force_prec=0 if args.prec == "fp64" else None)
    sch = Scheduler(eng, budget_bytes=int(args.budget_gib * (1 << 30)), round_steps=args.round_steps)
    out = sch.run(reqs, realtime=not args.virtual)
    fp64_lat = [j.finished_s - j.req.arrival_s for j in sch.finished
                if j.status == "done" and (eng._prec(j.req) == 0)]
    out.update({"mode": args.mode, "prec": args.prec, "requests": args.requests,
                "budget_bytes": int(args.budget_gib * (1 << 30)), "steps_scale": args.steps_scale,
                "fp64_subset": {"n": len(fp64_lat),
                                "p50_s": float(np.percentile(fp64_lat, 50)) if fp64_lat else None,
                                "p99_s": float(np.percentile(fp64_lat, 99)) if fp64_lat else None},
                "failed_fp32": sum(1 for j in sch.finished if j.status == "failed" and eng._prec(j.req) == 1),
                "failed_fp64": sum(1 for j in sch.finished if j.status == "failed" and eng._prec(j.req) == 0)})
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
