"""Write tests/golden/riemann_suite.json from the FP64 CPU oracle (no other source).

For the Riemann problems of Sec. 5.1 (Eqs. 21-23, 25) at the paper's dx, dt, tau and lambda,
it runs each to the paper's final time on a line wide enough that no wave reaches the ends,
then stores the L1 distance to the exact gamma = 2 solution and 32 sampled nodes of rho, u, p.
Run: python tests/golden/make_riemann_suite.py   (about 2-3 minutes on 4 cores)
"""
import json
import multiprocessing as mp
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

CASES = [("sod", 1000), ("lax", 2000), ("sjogreen", 400), ("collision", 3000)]


def run(case):
    import numpy as np
    from oracle import fdlbm as O
    from oracle import riemann
    from paper_0801_4169_gb300 import workloads as W
    name, nx = case
    w = W.riemann1d(name, nx=nx)
    s = O.Sim(w.nx, 1, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc)
    s.set_macro(*w.macros())
    rc = s.step(w.steps)
    r, u, v, T = [a[0] for a in s.get_macro()]
    x = (np.arange(nx) + 0.5) * w.dx
    L, R = w.meta["left"], w.meta["right"]
    re, ue, pe = riemann.sample((L[0], L[1], L[0] * L[3]), (R[0], R[1], R[0] * R[3]),
                                (x - w.meta["x0"]) / (w.steps * w.dt))
    idx = np.linspace(0, nx - 1, 32).round().astype(int)
    return name, {"nx": nx, "steps": w.steps, "rc": rc,
                  "l1_rho": float(np.mean(np.abs(r - re))), "l1_u": float(np.mean(np.abs(u - ue))),
                  "l1_p": float(np.mean(np.abs(r * T - pe))), "rho_min": float(r.min()),
                  "sample_index": idx.tolist(), "rho": r[idx].tolist(), "u": u[idx].tolist(),
                  "p": (r * T)[idx].tolist()}


if __name__ == "__main__":
    out = {"_about": "FP64 CPU oracle at the paper's Sec. 5.1 parameters; written by tests/golden/make_riemann_suite.py"}
    with mp.get_context("spawn").Pool(len(CASES)) as pool:
        for name, rec in pool.imap(run, CASES):
            out[name] = rec
            print(name, rec["rc"], rec["l1_rho"], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "riemann_suite.json"), "w") as fh:
        json.dump(out, fh, indent=1)
