"""Benchmark of the fused FDLBM step on GB300 (one JSON line on rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--prec fp32|fp64] [--impl reference]

A "step" is one time step of the whole method (moments -> f_eq -> Eq. 17 -> boundary fill) over
the workload's grid. The metric is GLUPS: site updates of all 33 velocities per second (nx*ny*steps/s).

Default workload: the 4096 x 4096 four-quadrant Riemann problem (FP32 f; moments summed exactly in
fixed point and finished in FP64; FP64 f_eq;
dx = 2.5e-4, dt = tau = 2.5e-6, lambda = 3, outflow on every side). Its f pair is 4.4 GB, far
above the 129 MB L2, so no L2 flush is needed between steps.

- value: device time over K steps from CUDA events on the solver's stream, with inputs already
  resident in HBM.
- e2e: the public call sequence with pinned host buffers inside the timed region:
  fdlbm_set_macro (H2D), fdlbm_step(K), fdlbm_get_macro (D2H).
- roofline: the fused step kernel against the FP64 pipe (2 FP64 instructions per clock per SM,
  the nominal 1.25 TFLOP/s). FP64 on this part issues ~60x slower than FP32, so the kernel is
  bound by FP64 issue, not HBM. The HBM figures are reported beside it.
- cpu_baseline: the FP64 CPU oracle, timed on a bounded sample of the same workload.

N > 1 (torchrun): every rank runs an independent replica with its own seed (weak scaling, no
data-path collective); the time is the max over ranks.

--workload vn_sec4 benchmarks the von Neumann tool instead (Sec. 4, Eqs. 18-20): a "step" is one
fdlbm_vn_spectrum call over every curve of Figs. 2, 4, 5 and 6 at 256 wave numbers (5632 33 x 33
complex eigenproblems in double-double). The metric is amplification-matrix spectra per second.
Its oracle is the 40-digit mpmath computation in oracle/vonneumann.py, because FP64 eigenvalues
are wrong at these states.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# FP64 arithmetic instructions (DADD + DFMA + DMUL) per site update, each node's moments counted
# once: ncu thread-level counts of the split step's two kernels, whose sum is the fused step's
# work without the moments of the tile ring (see profiles/). FP32 storage sums its moments in
# 64-bit fixed point on the integer pipes, hence the lower count (FP32 storage: 130 update +
# 15 moments; FP64: 481 + 89). FNEQ32: ncu's count of k_step_fneq per site (the equilibrium rebuilt
# on each tile's halo before the stencil and formed again from the new moments). fp32dw (the
# double-word equilibrium): 15 for the moments and 4 to split the macros into double words (ncu:
# 23.9 with the tile ring's moments).
FP64_OPS_PER_LUP = {"fp64": 570, "fp32": 145, "fneq32": 927, "fp32dw": 19}
# DRAM bytes (read + write) per site update of one step's launches (k_step, or k_moments +
# k_update), by (precision, tile variant): ncu dram__bytes_read.sum + dram__bytes_write.sum of one
# step of this bench's 4096^2 workload (single-pass capture), divided by the sites. Reported as roofline.traffic when the autotuner
# picks the captured variant, else null.
TRAFFIC_B_PER_SITE = {("fp32", 2): 268.5, ("fp32", 6): 267.6, ("fp32", 11): 467.8, ("fp64", 7): 836.7,
                      ("fp64", 10): 873.5, ("fp32dw", 6): 266.3, ("fp32dw", 12): 263.1}
# Warp instructions issued per site update (ncu smsp__inst_executed over the sites, 2048^2, same
# kernels), by (precision, tile variant): the double-word step binds on instruction issue, whose
# peak is 4 warp instructions per clock per SM (one per scheduler).
WARP_INST_PER_SITE = {("fp32", 6): 121.6, ("fp32dw", 6): 131.3, ("fp32dw", 12): 125.0}
ISSUE_PER_CLK_SM = 4.0
DTYPE = {"fp64": "f64", "fp32": "f32-store/fixed-point+f64-moments/f64-feq",
         "fneq32": "f64-macros+f32-fneq/f64-step", "fp32dw": "f32-store/df32-feq"}
# Variants that split a step into two launches (moment pass + update pass). Their minimum bytes per
# site update: f read twice and written once, the moment buffer (4 FP64 + P) written and read.
SPLIT_VARIANTS = (10, 11)
# Variants that run all the steps of a call in one cooperative launch (up to 4096 steps each).
PERSISTENT_VARIANTS = (13, 14)
GRAPH_VARIANT = 15  # the ring-parallel step launched from captured CUDA graphs
BYTES_PER_LUP_SPLIT = {"fp64": 3 * 33 * 8 + 2 * (4 * 8 + 8), "fp32": 3 * 33 * 4 + 2 * (4 * 8 + 4),
                       "fp32dw": 3 * 33 * 4 + 2 * (4 * 8 + 4)}
# Minimum HBM bytes per site update: read and write all 33 f once.
BYTES_PER_LUP = {"fp64": 2 * 33 * 8, "fp32": 2 * 33 * 4, "fneq32": 2 * (33 * 4 + 4 * 8), "fp32dw": 2 * 33 * 4}
# FP64 instructions (DADD + DFMA + DMUL) per amplification-matrix spectrum of the von Neumann
# tool on the Sec. 4 sweep: ncu thread-level counts of k_vn divided by the cases. They include the
# rotation parameters every lane computes alike, so they bound the algorithmic work from above.
FP64_OPS_PER_VN_MATRIX = 15.48e6
# FP64 issue peak: 2 instructions per clock per SM, i.e. the nominal 1.25 TFLOP/s at 2.07 GHz
# (ncu's pct-of-peak for the FP64 pipe agrees with it).
FP64_OPS_PER_CLK_SM = 2.0
N_SM = 152


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def make_workload(name, seed=0, small=False, n=None):
    from paper_0801_4169_gb300 import workloads as W
    if name == "riemann4096":
        return W.riemann4q(n=n or (256 if small else 4096), seed=seed)
    if name == "reflection1200x300":
        return W.reflection(nx=300, ny=75) if small else W.reflection()
    if name == "shock4000x4":
        return W.shock_tube(nx=400 if small else 4000)
    if name == "sod400x4":
        return W.sod()
    raise SystemExit("unknown workload %s" % name)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_over_ranks(ms_local, lups_local, dist=None, device=None):
    """Weak-scaling aggregation across replicas: the job's time is the slowest rank's, its work the
    sum over ranks. Works with any torch.distributed backend (NCCL on GPUs, gloo in the CPU tests)."""
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    w = torch.tensor([float(lups_local)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(w, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return ms, float(w.item()), float(w.item()) / (ms * 1e-3) / 1e9


def _oracle_case(name):
    from paper_0801_4169_gb300 import workloads as W
    if name == "riemann4096":
        return W.riemann4q(n=256, seed=0), "256x256 sub-grid of the four-quadrant problem (same dx, dt, states)"
    if name == "reflection1200x300":
        return W.reflection(nx=300, ny=75), "300x75 downscale of the reflection problem"
    if name == "shock4000x4":
        return W.shock_tube(nx=4000, ny=1), "4000x1 (y-uniform rows are identical)"
    return W.sod(ny=1), "400x1 (y-uniform rows are identical)"


def _oracle_replica(w, budget_s, out, k):
    """One oracle solve stepped until budget_s has passed; out[k] = (site updates, seconds)."""
    from oracle import fdlbm as O
    s = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
    s.set_macro(*w.macros())
    s.step(1)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        rc = s.step(5)
        steps += 5
        if rc:
            break
    out[k] = (w.nx * w.ny * steps, time.perf_counter() - t0)
    s.close()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample(name, budget_s=20.0):
    """Time the FP64 CPU oracle on a bounded sample of the workload (a sub-grid, a few steps).

    The oracle is single-threaded. It runs once alone (one core), then as one independent replica
    per host core in threads (ctypes releases the GIL during a call), which is the all-core
    throughput of the same program. value/cores report the all-core run; single_core the first."""
    import threading
    w, sample = _oracle_case(name)
    half = budget_s / 2.0
    one = [None]
    _oracle_replica(w, half, one, 0)
    ncore = host_cores()
    res = [None] * ncore
    th = [threading.Thread(target=_oracle_replica, args=(w, half, res, k)) for k in range(ncore)]
    t0 = time.perf_counter()
    for t in th:
        t.start()
    for t in th:
        t.join()
    wall = time.perf_counter() - t0
    lups_all = sum(r[0] for r in res)
    single = one[0][0] / one[0][1] / 1e9
    return {"value": lups_all / wall / 1e9, "unit": "GLUPS", "cores": ncore, "kind": "oracle",
            "sample": "%s; single-threaded FP64 C, %.1f s on one core, then %d replicas in %d threads for %.1f s"
                      % (sample, one[0][1], ncore, ncore, wall),
            "single_core": {"value": single, "unit": "GLUPS", "cores": 1}}


def vn_oracle_sample(budget_s=20.0):
    """The 40-digit oracle (mpmath) on the first cases of the Sec. 4 sweep, spread over its curves."""
    from oracle import vonneumann as V
    from paper_0801_4169_gb300 import workloads as W
    rows, curves, xi = W.vn_sec4_cases(nk=256)
    dx, dy, dt, tau = W.VN_SEC4_GRID
    order = np.arange(len(rows)).reshape(len(curves), len(xi)).T.ravel()  # one per curve, then the next k
    done = 0
    t0 = time.perf_counter()
    for i in order:
        r = rows[i]
        fl = int(r[7])
        V.max_abs_eig_mp(tuple(r[:4]), r[4], r[5], dx, dy, dt, tau, r[6], dps=40, lw=not fl & 1, disp=not fl & 2,
                         visc=not fl & 4)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "matrices/s", "cores": 1, "kind": "oracle",
            "sample": "%d of the %d Sec. 4 cases at 40 digits (mpmath), %.1f s single-threaded" % (done, len(rows), el)}


def posed_states_leg(F, torch, prec, variant, steps=20, warmup=3):
    """The 4096^2 four-quadrant step at the states first posed for it (rho in [0.1, 2], p in
    [0.03, 1.5], local Mach <= 10; seed 2, lambda = 3), same precision and tile variant, timed over
    the first steps: whether high-kappa states (far-apart exponents, rare conversions) cost
    throughput. The scheme rejects these states later in the run (every precision by step 2000),
    so the status after the timed steps is reported with the number."""
    from paper_0801_4169_gb300 import workloads as W
    w = W.riemann4q(n=4096, seed=2, lam=3.0, mach_max=10.0, rho_range=(0.1, 2.0), p_range=(0.03, 1.5))
    st = torch.cuda.Stream()
    s = F.Solver.from_workload(w, prec, stream=st)
    s.set_variant(variant)
    s.step(warmup)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.step(steps)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    try:
        status = s.sync()
    except F.FdlbmError as e:
        status = e.code
    s.close()
    return {"workload": w.name, "ranges": "rho [0.1, 2], p [0.03, 1.5], Mach <= 10, seed 2, lambda 3",
            "ms_per_step": ms, "glups": w.nx * w.ny / (ms * 1e-3) / 1e9, "steps": steps,
            "status_after": status}


def host_copy_rates(torch, h_src, h_dst):
    """This box's pinned host <-> device copy rates (GB/s, best of 3 copies of one macro array),
    taken before the end-to-end pass: the e2e figure's copies run at these rates, which differ
    between machines several-fold."""
    d = torch.empty(h_src.shape, dtype=h_src.dtype, device="cuda")
    nbytes = h_src.numel() * h_src.element_size()
    out = {}
    for name, dst, src in (("h2d", d, h_src), ("d2h", h_dst, d)):
        best = float("inf")
        for _ in range(3):
            torch.cuda.synchronize()
            t = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t)
        out[name] = round(nbytes / best / 1e9, 1)
    del d
    return out


def issue_roofline(prec_name, variant, site_rate, sm_mhz):
    """Instruction issue against its peak, where ncu's warp-instruction count for the variant is
    known (else null)."""
    ips = WARP_INST_PER_SITE.get((prec_name, variant))
    if ips is None:
        return None
    peak = ISSUE_PER_CLK_SM * N_SM * sm_mhz * 1e6 / 1e9
    achieved = ips * site_rate / 1e9
    return {"achieved": achieved, "peak": peak, "unit": "G warp instructions/s", "frac": achieved / peak,
            "warp_inst_per_site": ips,
            "peak_derivation": "4 warp instructions/clk/SM x 152 SMs x %.0f MHz sampled" % sm_mhz}


def df32_leg(F, torch, w, peaks, sm_mhz, steps=20, warmup=3):
    """The labelled double-word variant (FDLBM_FP32_STORE_DW, "f32-store/df32-feq") on the same
    workload: FP32 storage and fixed-point moments as the headline, the per-ring equilibrium
    constants and pairs in double-word FP32 on the FP32 pipe. Autotuned, timed like the headline."""
    st = torch.cuda.Stream()
    s = F.Solver.from_workload(w, F.FDLBM_FP32_STORE_DW, stream=st)
    times = s.autotune(3)
    variant = F.fdlbm_get_variant(s.h)
    s.step(warmup)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.step(steps)
    e1.record(st)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    status = s.sync()
    s.close()
    site_rate = w.nx * w.ny / (ms * 1e-3)
    split = variant in SPLIT_VARIANTS
    fp64_peak = FP64_OPS_PER_CLK_SM * N_SM * sm_mhz * 1e6 / 1e9
    fp64 = FP64_OPS_PER_LUP["fp32dw"] * site_rate / 1e9
    hbm = (BYTES_PER_LUP_SPLIT if split else BYTES_PER_LUP)["fp32dw"] * site_rate / 1e9
    return {"dtype": DTYPE["fp32dw"], "value": site_rate / 1e9, "unit": "GLUPS", "ms_per_step": ms,
            "tile_variant": variant, "kernel": "k_step_tma (tile by tensor copy)" if variant == 12 else "k_step",
            "autotune_ms": [round(t, 4) for t in times], "status": status,
            "fp64_pipe": {"achieved": fp64, "peak": fp64_peak, "unit": "G FP64-pipe ops/s", "frac": fp64 / fp64_peak},
            "hbm": {"achieved_gbs": hbm, "peak_gbs": peaks.get("hbm_gbs"), "frac": hbm / peaks.get("hbm_gbs", 6800.0)},
            "issue": issue_roofline("fp32dw", variant, site_rate, sm_mhz),
            "traffic": (TRAFFIC_B_PER_SITE.get(("fp32dw", variant), 0) * w.nx * w.ny or None)
            if (w.nx, w.ny) == (4096, 4096) else None,
            "error_vs_fp64_path": "4096^2, 2000 steps, seeds 0-2: L1(rho) 1.81e-7, 4.32e-7, 8.71e-7 and "
                                  "max |d rho|/max rho 7.3e-6, 8.6e-6, 7.5e-6 (bounds 1e-6 and 1e-5, "
                                  "tests/test_gpu_parity.py::test_fp32_storage_error_at_full_size)"}


def serving_leg(n_req=64, steps_scale=0.25, seed=0, budget_bytes=1 << 30):
    """The continuous-batching runtime on a seeded stream of shock-tube solves (the serving
    workload's recipe: Poisson arrivals at 200 requests/s, nx ~ U{256..16384}, ny = 4,
    Ms ~ U[2, 10], steps ~ U{2000..20000}, here n_req requests with steps scaled by steps_scale).

    Three runs of the same stream: batched FP64, one launch sequence per solve in FP64 (the
    baseline), and batched with the requests drawn as FP32 in FNEQ32. The FNEQ32 requests' results
    are compared with the same requests' FP64 results."""
    from paper_0801_4169_gb300 import fdlbm as F
    from paper_0801_4169_gb300 import serve
    from paper_0801_4169_gb300 import workloads as W
    reqs = W.serving_requests(n=n_req, seed=seed)
    for r in reqs:
        r.steps = max(1, int(round(r.steps * steps_scale)))
    warm = W.serving_requests(n=4, seed=seed + 1)
    for r in warm:
        r.steps = 40
    runs = (("batched_fp64", "gpu", 0, F.FDLBM_FP32_STORE), ("per_solve_fp64", "separate", 0, F.FDLBM_FP32_STORE),
            ("batched_mixed_fneq32", "gpu", None, F.FDLBM_FNEQ32))
    res, outs = {}, {}
    for name, engine, override, fp32_as in runs:
        srv = serve.Server(budget_bytes=budget_bytes, engine=engine)
        serve.replay(srv, warm, realtime=False, prec_override=override, fp32_as=fp32_as)
        srv.close()
        srv = serve.Server(budget_bytes=budget_bytes, engine=engine)
        out, st = serve.replay(srv, reqs, prec_override=override, fp32_as=fp32_as)
        srv.close()
        outs[name] = {r.rid: (r, status, m) for (r, status, m, secs, err) in out.values()}
        res[name] = {k: st[k] for k in ("aggregate_glups", "p50_s", "p99_s", "mean_s", "wall_s", "done", "failed",
                                         "max_active", "rounds")}
    errs = []
    for rid, (r, status, m) in outs["batched_mixed_fneq32"].items():
        ref = outs["batched_fp64"].get(rid)
        if r.prec != 1 or status != F.FDLBM_REQ_DONE or ref is None or ref[1] != F.FDLBM_REQ_DONE:
            continue
        a, b = m[0], ref[2][0]
        errs.append((float(np.mean(np.abs(a - b)) / np.mean(np.abs(b))), float(np.max(np.abs(a - b)) / np.max(np.abs(b)))))
    e = np.array(errs) if errs else np.zeros((0, 2))
    res["fneq32_vs_fp64"] = {"requests": len(errs),
                             "l1_rho_median": float(np.median(e[:, 0])) if len(e) else None,
                             "l1_rho_max": float(e[:, 0].max()) if len(e) else None,
                             "max_rho_rel_max": float(e[:, 1].max()) if len(e) else None}
    res["recipe"] = ("%d requests (seed %d), Poisson arrivals at 200/s, nx ~ U{256..16384}, ny = 4, Ms ~ U[2, 10] "
                     "with the upstream at -(Ms - 2) c1, steps ~ U{2000..20000} x %g, precision ~ Bernoulli(1/2) "
                     "(FP32 requests as FNEQ32 in the mixed run), HBM budget %d MiB, lambda = 2"
                     % (n_req, seed, steps_scale, budget_bytes >> 20))
    res["speedup_batched_vs_per_solve"] = (res["batched_fp64"]["aggregate_glups"] /
                                           res["per_solve_fp64"]["aggregate_glups"])
    return res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.workload == "vn_sec4":
        cb = vn_oracle_sample(budget_s=max(5.0, min(60.0, 4.0 * args.steps)))
        line = {"impl": "reference", "metric": "amplification-matrix spectra/s", "value": cb["value"],
                "unit": "matrices/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "mp40",
                "data": "synthetic", "config": {"workload": "vn_sec4", "impl": "40-digit oracle (oracle/vonneumann.py)"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    cb = oracle_sample(args.workload, budget_s=max(5.0, min(60.0, 4.0 * args.steps)))
    line = {"impl": "reference", "metric": "GLUPS", "value": cb["value"], "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "impl": "FP64 CPU oracle (oracle/fdlbm_oracle.c)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_vn(args, F, torch, dist, rank, local, world):
    """The von Neumann tool on the Sec. 4 sweep (see the module docstring)."""
    from paper_0801_4169_gb300 import workloads as W
    rows, curves, xi = W.vn_sec4_cases(nk=256)
    dx, dy, dt, tau = W.VN_SEC4_GRID
    cases = F.vn_cases(rows[:, :4], rows[:, 4], rows[:, 5], rows[:, 6], rows[:, 7].astype(np.int32))
    n = len(cases)
    stream = torch.cuda.Stream()
    raw = cases.view(np.uint8)
    h_cases = torch.empty(raw.shape, dtype=torch.uint8, pin_memory=True)
    h_cases.numpy()[...] = raw
    h_max = torch.empty(n, dtype=torch.float64, pin_memory=True)
    with torch.cuda.stream(stream):
        d_cases = h_cases.to("cuda", non_blocking=True)
        d_max = torch.empty(n, dtype=torch.float64, device="cuda")
        d_st = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        F.fdlbm_vn_spectrum(d_cases, n, dx, dy, dt, tau, d_max, None, None, d_st, stream)
    stream.synchronize()
    sampler = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0.record(stream)
    for _ in range(args.steps):
        F.fdlbm_vn_spectrum(d_cases, n, dx, dy, dt, tau, d_max, None, None, d_st, stream)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    st = d_st.cpu().numpy()
    if dist:
        dist.barrier()
    ms_max, work, _ = aggregate_over_ranks(ms, n * args.steps, dist, device="cuda")
    rate = work / (ms_max * 1e-3)
    # end to end: pinned host cases in, max |omega| out, every step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            d_cases.copy_(h_cases, non_blocking=True)
        F.fdlbm_vn_spectrum(d_cases, n, dx, dy, dt, tau, d_max, None, None, d_st, stream)
        with torch.cuda.stream(stream):
            h_max.copy_(d_max, non_blocking=True)
        stream.synchronize()
    t_e2e = time.perf_counter() - t0
    t_e2e_max, e2e_work, _ = aggregate_over_ranks(t_e2e * 1e3, n * args.steps, dist, device="cuda")
    e2e_rate = e2e_work / (t_e2e_max * 1e-3)
    peaks, peak_kind = load_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = FP64_OPS_PER_CLK_SM * N_SM * sm_mhz * 1e6 / 1e9
    per_launch_rate = n / (ms / args.steps * 1e-3)
    achieved = FP64_OPS_PER_VN_MATRIX * per_launch_rate / 1e9 if FP64_OPS_PER_VN_MATRIX else None
    line = {
        "metric": "amplification-matrix spectra/s", "value": rate, "unit": "matrices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64x2 (double-double)", "data": "synthetic",
        "config": {"workload": "vn_sec4", "cases": n, "curves": len(curves), "nk": len(xi),
                   "l2": "inputs of %d KB: every step reads the same cases (compute-bound, no flush)" % (raw.size // 1024),
                   "status_counts": np.bincount(st, minlength=3).tolist(), "parallelism": "replicas%d" % world},
        "roofline": {"bound": "alu", "kernel": "k_vn", "achieved": achieved, "peak": fp64_peak,
                     "unit": "G FP64-pipe ops/s", "frac": achieved / fp64_peak if achieved else None, "traffic": None,
                     "peak_derivation": "2 FP64 ops/clk/SM (nominal 1.25 TFLOP/s) x 152 SMs x %.0f MHz sampled" % sm_mhz},
        "clocks": clocks,
        "e2e": {"value": e2e_rate, "unit": "matrices/s", "h2d_bytes_per_step": int(raw.size),
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = vn_oracle_sample(budget_s=20.0)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="riemann4096",
                    choices=["riemann4096", "reflection1200x300", "shock4000x4", "sod400x4", "vn_sec4"])
    ap.add_argument("--prec", default=None, choices=["fp32", "fp64", "fneq32", "fp32dw"])
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving leg")
    ap.add_argument("--small", action="store_true", help="a small version of the workload (profiling)")
    ap.add_argument("--n", type=int, default=None, help="grid edge of the four-quadrant workload (profiling)")
    ap.add_argument("--variant", type=int, default=None,
                    help="launch variant instead of the autotuner's choice (profiling: ncu's per-launch overhead "
                         "biases the autotuner against two-launch variants)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_0801_4169_gb300 import fdlbm as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.workload == "vn_sec4":
        run_vn(args, F, torch, dist, rank, local, world)
        if dist:
            dist.destroy_process_group()
        return
    prec_name = args.prec or ("fp64" if args.workload == "sod400x4" else "fp32")
    prec = {"fp64": F.FDLBM_FP64, "fp32": F.FDLBM_FP32_STORE, "fneq32": F.FDLBM_FNEQ32,
            "fp32dw": F.FDLBM_FP32_STORE_DW}[prec_name]

    w = make_workload(args.workload, seed=rank, small=args.small, n=args.n)
    stream = torch.cuda.Stream()
    solver = F.Solver(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, prec, 0, w.bstate, stream=stream)
    # pinned host copies of the inputs (for the end-to-end leg)
    pinned, pinned_t = [], []
    for a in w.macros():
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        pinned_t.append(t)
        pinned.append(t.numpy())
    solver.set_macro(*pinned)
    if args.variant is None:
        times = solver.autotune(3)
    else:
        solver.set_variant(args.variant)
        times = []
    variant = F.fdlbm_get_variant(solver.h)
    solver.step(args.warmup)
    solver.sync()

    sampler = ClockSampler(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    e0.record(stream)
    solver.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    status = solver.sync()
    lups = w.nx * w.ny * args.steps
    if dist:
        dist.barrier()
    ms_max, lups_all, glups = aggregate_over_ranks(ms, lups, dist, device="cuda")
    per_launch_ms = ms / args.steps

    # end-to-end: the public API with pinned host buffers, copies inside the timed region
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    h_out_t = [torch.empty(a.shape, dtype=torch.float64, pin_memory=True) for a in w.macros()]
    h_out = [t.numpy() for t in h_out_t]
    host_copy = host_copy_rates(torch, pinned_t[0], h_out_t[0])
    # one untimed pass through the same calls and pinned buffers, as the steps get warm-up steps:
    # the first DMA touch of pinned pages can cost several times the copy on a host whose memory
    # earlier processes churned (its parts are reported as warmup_parts_ms)
    tw0 = time.perf_counter()
    solver.set_macro(*pinned)
    tw1 = time.perf_counter()
    F.lib().fdlbm_get_macro(solver.h, *[F._hp(a) for a in h_out])
    tw2 = time.perf_counter()
    warm_parts = {"set_macro": round((tw1 - tw0) * 1e3, 2), "get_macro": round((tw2 - tw1) * 1e3, 2)}
    # three timed passes, each a whole solve through the public calls with its copies; the line
    # reports the median pass (host copies on these machines stall now and then for tens of ms)
    passes = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.set_macro(*pinned)                      # synchronous: H2D copies and f = f_eq
        t1 = time.perf_counter()
        solver.step(args.steps)
        solver.sync()                                  # get_macro would wait for the steps anyway
        t2 = time.perf_counter()
        rc = F.lib().fdlbm_get_macro(solver.h, *[F._hp(a) for a in h_out])
        t3 = time.perf_counter()
        passes.append((t3 - t0, t0, t1, t2, t3, rc))
    t_e2e, t0, t1, t2, t3, rc = sorted(passes)[1]
    rc = next((p[5] for p in passes if p[5]), 0)  # the first failing pass's status, if any
    _, _, e2e_glups = aggregate_over_ranks(t_e2e * 1e3, lups, dist, device="cuda")
    macro_bytes = 4 * w.nx * w.ny * 8

    peaks, peak_kind = load_peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp64_peak = FP64_OPS_PER_CLK_SM * N_SM * sm_mhz * 1e6 / 1e9  # G ops/s at the sampled clock
    # the same pipe measured on this GPU now: independent FMA chains at full occupancy
    fp64_measured = F.fdlbm_fp64_rate(20000, stream) / 1e9
    site_rate = w.nx * w.ny / (per_launch_ms * 1e-3)
    achieved = FP64_OPS_PER_LUP[prec_name] * site_rate / 1e9
    split = variant in SPLIT_VARIANTS
    hbm_gbs = (BYTES_PER_LUP_SPLIT if split else BYTES_PER_LUP)[prec_name] * site_rate / 1e9
    tb = TRAFFIC_B_PER_SITE.get((prec_name, variant)) if (w.nx, w.ny) == (4096, 4096) else None
    traffic = tb * w.nx * w.ny if tb else None

    line = {
        "metric": "GLUPS", "value": glups, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE[prec_name],
        "data": "synthetic",
        "config": {"workload": w.name, "nx": w.nx, "ny": w.ny, "precision": prec_name,
                   "tile_variant": variant, "autotune_ms": [round(t, 4) for t in times],
                   "l2": "inputs larger than L2 (f pair %.2f GB)" % (BYTES_PER_LUP[prec_name] * w.nx * w.ny / 1e9)
                   if w.nx * w.ny * 33 * 4 > 129e6 else "inputs smaller than L2: steps read a warm cache",
                   "status": status, "parallelism": "replicas%d" % world},
        "roofline": {"bound": "alu", "kernel": "k_step_fneq (FNEQ32 step)" if prec_name == "fneq32" else
                     "k_moments + k_update (split step)" if split else
                     "k_step_tma (fused step, tile by tensor copy)" if variant == 12 and prec_name in ("fp32", "fp32dw")
                     else "k_persist_rp / k_persist_tile (persistent steps)" if variant in PERSISTENT_VARIANTS
                     and prec_name in ("fp32", "fp64")
                     else "k_step_rp (ring-parallel steps replayed from CUDA graphs of 32)" if variant == GRAPH_VARIANT
                     and prec_name in ("fp32", "fp64") else "k_step (fused step)",
                     "achieved": achieved,
                     "peak": fp64_peak, "unit": "G FP64-pipe ops/s", "frac": achieved / fp64_peak,
                     "traffic": traffic, "traffic_unit": "bytes per step (ncu DRAM read + write of its launches)",
                     "peak_derivation": "2 FP64 ops/clk/SM (nominal 1.25 TFLOP/s) x 152 SMs x %.0f MHz sampled" % sm_mhz,
                     "peak_measured": fp64_measured, "frac_of_measured": achieved / fp64_measured,
                     "peak_measured_how": "fdlbm_fp64_rate: 8 independent FMA chains per thread, 8 CTAs x 256 "
                                          "threads per SM, CUDA events, right after the timed steps",
                     "hbm": {"achieved_gbs": hbm_gbs, "peak_gbs": peaks.get("hbm_gbs"), "peak_kind": peak_kind,
                             "frac": hbm_gbs / peaks.get("hbm_gbs", 6800.0)},
                     "issue": issue_roofline(prec_name, variant, site_rate, sm_mhz)},
        "clocks": clocks,
        "e2e": {"value": e2e_glups, "unit": "GLUPS", "h2d_bytes_per_step": macro_bytes / args.steps,
                "d2h_bytes_per_step": macro_bytes / args.steps, "status": int(rc),
                "note": "one solve per timed region: set_macro (H2D) + %d steps + get_macro (D2H); the median of "
                        "3 passes after an untimed one" % args.steps,
                "passes_ms": [round(p[0] * 1e3, 2) for p in passes],
                "parts_ms": {"set_macro": round((t1 - t0) * 1e3, 2), "steps": round((t2 - t1) * 1e3, 2),
                             "get_macro": round((t3 - t2) * 1e3, 2)},
                "host_copy_gbs": host_copy, "warmup_parts_ms": warm_parts},
        "gpu_launches": -(-args.steps // 4096) if variant in PERSISTENT_VARIANTS and prec_name in ("fp32", "fp64")
        else args.steps * (2 if split else 1),
    }
    solver.close()
    if rank == 0 and world == 1 and args.workload == "riemann4096" and not args.small and args.n is None:
        line["posed_states"] = posed_states_leg(F, torch, prec, variant)
        if prec_name == "fp32":
            line["variant_df32"] = df32_leg(F, torch, w, peaks, sm_mhz)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(args.workload, budget_s=20.0)
    if rank == 0 and world == 1 and not args.no_serving and args.workload == "riemann4096" and not args.small:
        line["serving"] = serving_leg()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
