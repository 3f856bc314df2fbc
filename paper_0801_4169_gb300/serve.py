"""Serving FDLBM solves with the library's continuous-batching runtime (fdlbm_server_*).

The runtime lives in the library (csrc/fdlbm_server.cu): a worker thread admits requests by HBM
budget and slots in submission order, advances all admitted solves together, one batch per
scheme group with one kernel launch per time step, and retires them with their time to
solution. This module only wraps that ABI and replays a request stream (W.serving_requests):
each request is submitted at its arrival time, and every outcome is collected at the end.

    python -m paper_0801_4169_gb300.serve --requests 512 [--engine gpu|separate] [--prec mixed|fp64]
        [--fp32-as store|fneq]

engine "separate" is the baseline: the same scheduler, every solve stepped by its own launches.
"""
import argparse
import json
import time

import numpy as np

from . import fdlbm as F
from . import workloads as W

ENGINES = {"gpu": F.FDLBM_ENGINE_GPU, "separate": F.FDLBM_ENGINE_GPU_SEPARATE, "sim": F.FDLBM_ENGINE_SIMULATED}


class Server:
    """Thin wrapper over fdlbm_server_*: submit workloads, wait, collect results and statistics."""

    def __init__(self, budget_bytes=1 << 30, max_slots=256, round_steps=500, engine="gpu", stream=None):
        self.h = F.fdlbm_server_create(budget_bytes, max_slots, round_steps, ENGINES[engine], stream)
        self.shapes = {}

    def submit(self, w, steps, prec, sim_fail_step=0):
        cfg = F.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, prec)
        rid = F.fdlbm_server_submit(self.h, cfg, *w.macros(), steps, bstate=w.bstate, sim_fail_step=sim_fail_step)
        self.shapes[rid] = (w.nx, w.ny)
        return rid

    def poll(self, rid):
        return F.fdlbm_server_poll(self.h, rid)

    def wait(self, rid, timeout_s=-1.0):
        return F.fdlbm_server_wait(self.h, rid, timeout_s)

    def result(self, rid):
        """(status, (rho, u, v, T) or None, seconds to solution or None, error message)."""
        nx, ny = self.shapes.pop(rid)
        try:
            rho, u, v, T, secs = F.fdlbm_server_result(self.h, rid, nx, ny)
            return F.FDLBM_REQ_DONE, (rho, u, v, T), secs, ""
        except F.FdlbmError as e:
            return F.FDLBM_REQ_FAILED, None, None, str(e)

    def stats(self):
        return F.fdlbm_server_stats(self.h)

    def close(self):
        if self.h:
            F.fdlbm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def replay(server, requests, lam=2.0, realtime=True, prec_override=None, fp32_as=F.FDLBM_FP32_STORE):
    """Submit each request at its arrival time (wall clock), then wait for all of them.

    A request drawn as FP32 storage runs in precision fp32_as (FDLBM_FP32_STORE, or FDLBM_FNEQ32,
    which stores f's departure from equilibrium); prec_override runs every request in one precision.
    Returns {rid: (request, status, macros, seconds, error)} and the server statistics."""
    t0 = time.perf_counter()
    ids = []
    for r in sorted(requests, key=lambda q: q.arrival_s):
        if realtime:
            delay = r.arrival_s - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
        w = W.request_workload(r, lam=lam)
        prec = (fp32_as if r.prec == 1 else F.FDLBM_FP64) if prec_override is None else prec_override
        ids.append((server.submit(w, r.steps, prec), r))
    out = {}
    for rid, r in ids:
        server.wait(rid)
        status, macros, secs, err = server.result(rid)
        out[rid] = (r, status, macros, secs, err)
    return out, server.stats()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--engine", default="gpu", choices=["gpu", "separate"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp32-as", default="store", choices=["store", "fneq"],
                    help="precision of the requests drawn as FP32: FP32 storage of f, or FNEQ32")
    ap.add_argument("--budget-gib", type=float, default=1.0)
    ap.add_argument("--round-steps", type=int, default=500)
    ap.add_argument("--steps-scale", type=float, default=1.0, help="scale every request's step count")
    args = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    reqs = W.serving_requests(n=args.requests, seed=args.seed)
    for r in reqs:
        r.steps = max(1, int(round(r.steps * args.steps_scale)))
    srv = Server(budget_bytes=int(args.budget_gib * (1 << 30)), round_steps=args.round_steps, engine=args.engine)
    fp32_as = F.FDLBM_FNEQ32 if args.fp32_as == "fneq" else F.FDLBM_FP32_STORE
    out, st = replay(srv, reqs, prec_override=0 if args.prec == "fp64" else None, fp32_as=fp32_as)
    srv.close()
    prec_of = lambda r: 0 if args.prec == "fp64" else r.prec  # noqa: E731
    fp64_lat = [secs for (r, status, m, secs, e) in out.values() if status == F.FDLBM_REQ_DONE and prec_of(r) == 0]
    st.update({"engine": args.engine, "prec": args.prec, "requests": args.requests,
               "budget_bytes": int(args.budget_gib * (1 << 30)), "steps_scale": args.steps_scale,
               "fp64_subset": {"n": len(fp64_lat),
                               "p50_s": float(np.percentile(fp64_lat, 50)) if fp64_lat else None,
                               "p99_s": float(np.percentile(fp64_lat, 99)) if fp64_lat else None},
               "failed_fp32": sum(1 for (r, s_, m, x, e) in out.values() if s_ != F.FDLBM_REQ_DONE and prec_of(r) == 1),
               "failed_fp64": sum(1 for (r, s_, m, x, e) in out.values() if s_ != F.FDLBM_REQ_DONE and prec_of(r) == 0)})
    print(json.dumps(st), flush=True)


if __name__ == "__main__":
    main()
