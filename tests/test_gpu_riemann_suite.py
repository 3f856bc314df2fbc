"""The Riemann problems of Sec. 5.1 on the GPU at the paper's parameters, to the paper's final time.

Each FP64 run is compared with the oracle's run of the same problem (tests/golden/riemann_suite.json,
written by tests/golden/make_riemann_suite.py from oracle/ only):
- 32 sampled nodes of rho, u, p agree to max(1e-9, 4 eps kappa sqrt(steps)) relative, with
  kappa = sum|f_eq|/n of the worse initial state. The two sides differ in summation order and FMA
  contraction; each step adds rounding of relative size ~eps kappa, and the differences
  accumulate like a random walk over 1800-20000 steps (kappa is 1.1e8 on the left of the
  collision problem);
- the L1 distance to the exact gamma = 2 solution is the oracle's to 1%.
Colella's problem (Eq. 24) is rejected by the scheme at its second step (T ratio 1e5); the GPU path
reports it like the oracle.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fdlbm as O  # noqa: E402
from oracle import riemann  # noqa: E402
from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402

def _gold():
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "riemann_suite.json")))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    F.lib()


@pytest.mark.parametrize("name", ["sod", "lax", "sjogreen", "collision"])
def test_riemann_problem_matches_oracle_at_final_time(name):
    g = _gold()[name]
    w = W.riemann1d(name, nx=g["nx"])
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    s.step(w.steps)
    rho, u, v, T = [a[0] for a in s.get_macro()]
    p = rho * T
    idx = np.array(g["sample_index"])
    kappa = max(np.abs(O.feq(*st)).sum() / st[0] for st in (w.meta["left"], w.meta["right"]))
    tol = max(1e-9, 4 * np.finfo(float).eps * kappa * np.sqrt(w.steps))
    for got, ref in ((rho[idx], g["rho"]), (u[idx], g["u"]), (p[idx], g["p"])):
        ref = np.array(ref)
        assert np.max(np.abs(got - ref)) <= tol * max(1.0, np.abs(ref).max())
    x = (np.arange(w.nx) + 0.5) * w.dx
    L, R = w.meta["left"], w.meta["right"]
    re, ue, pe = riemann.sample((L[0], L[1], L[0] * L[3]), (R[0], R[1], R[0] * R[3]),
                                (x - w.meta["x0"]) / (w.steps * w.dt))
    assert np.mean(np.abs(rho - re)) == pytest.approx(g["l1_rho"], rel=0.01)
    assert rho.min() > 0  # positivity (the paper's claim for the Sjogreen problem)


def test_colella_is_rejected_like_the_oracle():
    w = W.riemann1d("colella", nx=400, steps=3)
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    s.step(1)
    assert s.sync() == 0
    s.step(1)
    with pytest.raises(F.FdlbmError) as ei:
        s.sync()
    assert ei.value.code == F.FDLBM_E_NUMERIC
    o = O.Sim(w.nx, 1, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc)
    o.set_macro(*w.macros())
    assert o.step(1) == 0 and o.step(1) == -4


def _oracle_rounding_spread(w, flags, ulps=4.0, seed=0):
    """How far the oracle moves from its own result when every step's f is perturbed by up to
    `ulps` units in the last place (relative, independent per value): the spread that different
    rounding orders can produce once the shocks' nonlinear switch amplifies them."""
    a = O.Sim(w.nx, 1, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, flags=flags)
    a.set_macro(*w.macros())
    assert a.step(w.steps) == 0
    b = O.Sim(w.nx, 1, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, flags=flags)
    b.set_macro(*w.macros())
    rng = np.random.default_rng(seed)
    for _ in range(w.steps):
        b.step(1)
        f = b.get_f()
        b.set_f(f * (1 + ulps * np.finfo(float).eps * rng.uniform(-1, 1, f.shape)))
    ref = a.get_macro()[0][0]
    return ref, np.max(np.abs(b.get_macro()[0][0] - ref))


@pytest.mark.parametrize("flags", [0, F.FDLBM_NO_DISP])
def test_fig3_tube_matches_oracle_and_dispersion_damps_oscillations(flags):
    """Sec. 4, Fig. 3 tube on the GPU, with and without line III of Eq. 17.
    - GPU and oracle agree to 3x the oracle's own spread under 4-ulp per-step perturbations. After
      3000 steps the two shocks amplify rounding-order differences well beyond the kappa random
      walk (kappa = 1.7e4): the GPU differs by 1.6e-7, the spread is 1.8e-7 to 4.2e-7.
    - The dispersion line lowers the total variation of rho."""
    w = W.riemann1d("fig3", nx=400)
    res = {}
    for fl in (0, F.FDLBM_NO_DISP):
        s = F.Solver(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, F.FDLBM_FP64, fl, w.bstate)
        s.set_macro(*w.macros())
        s.step(w.steps)
        res[fl] = s.get_macro()[0][0]
    ref, spread = _oracle_rounding_spread(w, flags)
    assert np.max(np.abs(res[flags] - ref)) <= 3.0 * spread
    tv = {fl: np.abs(np.diff(r)).sum() for fl, r in res.items()}
    assert tv[0] < 0.97 * tv[F.FDLBM_NO_DISP]


def _front(rho, x, rho1, rho2, dx):
    """Position where rho falls through the mean of the jump (linear between nodes)."""
    half = 0.5 * (rho1 + rho2)
    i = np.where(rho > half)[0].max()
    return x[i] + (rho[i] - half) / (rho[i] - rho[i + 1]) * dx


@pytest.mark.parametrize("prec", [F.FDLBM_FP64, F.FDLBM_FNEQ32])
def test_strong_tube_at_full_size_against_rankine_hugoniot(prec):
    """The 4000 x 4 Mach-10 tube (normal Mach 10 into a counter-stream at -6 c1, lambda = 2), 5000
    steps, against the gamma = 2 Rankine-Hugoniot jump of the same shock (Sec. 5.1 states, m = 1):
    - the plateau between contact and shock: pressure within 0.5% of RH (measured -0.15%), velocity
      within 2% (+0.9%), density within 6% (+4.4%);
    - the shock speed, from the front at steps 2500 and 5000, is 15% above RH (4.60 against 4.00):
      line IV of Eq. 17 puts a node-wise coefficient outside the second difference, so it is not
      conservative, and at lambda = 2 it moves a Mach-10 shock this much. The bound keeps the speed
      within [1.10, 1.20] x RH;
    - FP64 storage and FNEQ32 give the same speed and plateau to 1e-5."""
    w = W.shock_tube(nx=4000, ny=4)
    rho2, u2, _, T2 = w.meta["post"]
    x = (np.arange(w.nx) + 0.5) * w.dx
    s = F.Solver.from_workload(w, prec)
    pos = []
    for _ in range(2):
        s.step(2500)
        rho, u, v, T = s.get_macro()
        for j in range(1, w.ny):
            assert np.array_equal(rho[j], rho[0])
        pos.append(_front(rho[0], x, 1.0, rho2, w.dx))
    speed = (pos[1] - pos[0]) / (2500 * w.dt)
    assert 1.10 * w.meta["W_lab"] <= speed <= 1.20 * w.meta["W_lab"]
    t = 5000 * w.dt
    a = int((w.meta["x0"] + u2 * t) / w.dx) + 10
    b = int(pos[1] / w.dx) - 10
    assert b - a > 100
    assert np.mean(rho[0][a:b] * T[0][a:b]) == pytest.approx(rho2 * T2, rel=5e-3)
    assert np.mean(u[0][a:b]) == pytest.approx(u2, rel=2e-2)
    assert np.mean(rho[0][a:b]) == pytest.approx(rho2, rel=6e-2)
    assert speed == pytest.approx(4.598336, rel=1e-5)
