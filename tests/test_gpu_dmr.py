"""Double Mach reflection (Sec. 5.2.2) on the GPU: moving boundary segments against the oracle.

The Eq. 27 data (Ms = 20 into gas at rest) are rejected by the scheme in exact arithmetic
(test_oracle_rejections.py); the paper's geometry and boundaries run at Ms = 6 (lambda = 20). The
GPU path applies the top boundary's moving Dirichlet segment and the bottom's Dirichlet stretch
before the wall after every step (fdlbm_set_boundary_segment), with the new state's time.
Tolerances: FP64 against the FP64 oracle as the other FP64 parity tests (summation order and FMA
contraction only); FP32 storage and FNEQ32 against the oracle are stated.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fdlbm as O  # noqa: E402
from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    F.lib()


def _oracle(w, steps):
    s = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
    for seg in w.meta["segments"]:
        s.set_segment(*seg)
    s.set_macro(*w.macros())
    assert s.step(steps) == 0
    return s


def _status(s):
    try:
        return s.sync()
    except F.FdlbmError as e:
        return e.code


def _reduced():
    return W.dmr(Ms=6.0, nx=125, ny=50, dx=4e-3, dt=4e-5)


def test_dmr_fp64_matches_oracle_with_ghost_rows():
    """Reduced DMR (125 x 50), 300 steps, FP64: every f of the interior and of the ghost rows
    above and below it within 1e-10 of max|f| of the oracle (the segments' f_eq differ from the
    oracle's in rounding only)."""
    w = _reduced()
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    s.step(300)
    fg = s.get_f_region(0, -2, w.nx, w.ny + 4)
    assert _status(s) == 0
    fo = _oracle(w, 300).get_f_padded()[:, :, 2:2 + w.nx]
    assert np.max(np.abs(fg - fo)) <= 1e-10 * np.abs(fo).max()


@pytest.mark.parametrize("prec,tol", [(F.FDLBM_FP32_STORE, 1e-2), (F.FDLBM_FNEQ32, 5e-6)])
def test_dmr_reduced_precisions_against_oracle(prec, tol):
    """The same run in FP32 storage and in FNEQ32: rho, u, v, T within the stated bound (max
    relative to each field's maximum) of the FP64 oracle. Measured: FP32 storage 4.4e-3 - 6.5e-3,
    FNEQ32 1.2e-6 - 2.1e-6 (FP64 storage: 3e-11 - 6e-11)."""
    w = _reduced()
    s = F.Solver.from_workload(w, prec)
    s.step(300)
    got = s.get_macro()
    assert _status(s) == 0
    ref = _oracle(w, 300).get_macro()
    for a, b in zip(got, ref):
        assert np.max(np.abs(a - b)) <= tol * np.max(np.abs(b))


def test_dmr_segments_are_applied_at_each_step():
    """Stepping 1 + 1 + ... gives the same bits as one call of the same steps (the segment is
    applied with the time of each new state), and clearing the top segment changes the result."""
    w = _reduced()
    a = F.Solver.from_workload(w, F.FDLBM_FP64)
    a.step(40)
    b = F.Solver.from_workload(w, F.FDLBM_FP64)
    for _ in range(40):
        b.step(1)
    fa = a.get_f_region(0, -2, w.nx, w.ny + 4)
    assert np.array_equal(fa, b.get_f_region(0, -2, w.nx, w.ny + 4))
    c = F.Solver.from_workload(w, F.FDLBM_FP64)
    F.fdlbm_clear_boundary_segment(c.h, 3)
    c.step(40)
    assert not np.array_equal(fa, c.get_f_region(0, -2, w.nx, w.ny + 4))


def test_segment_arguments_are_checked():
    w = W.sod(nx=32, ny=4)
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    for args in ((2, 0.1, 0.0, 1, 1.0, 0.0, 0.0, 1.0),        # periodic side
                 (0, float("nan"), 0.0, 1, 1.0, 0.0, 0.0, 1.0),
                 (0, 0.1, 0.0, 1, -1.0, 0.0, 0.0, 1.0)):
        with pytest.raises(F.FdlbmError) as ei:
            F.fdlbm_set_boundary_segment(s.h, *args)
        assert ei.value.code == F.FDLBM_E_ARG
    F.fdlbm_set_boundary_segment(s.h, 0, 0.1, 0.0, 1, 1.0, 0.0, 0.0, 1.0)
    b = F.fdlbm_batch_create()
    with pytest.raises(F.FdlbmError):
        F.fdlbm_batch_add(b, s.h)
    F.fdlbm_batch_destroy(b)


def test_dmr_full_size_at_mach_6():
    """The paper's grid (500 x 200, dx = 1e-3, dt = tau = 1e-5, lambda = 20) at Ms = 6, until the
    incident shock has moved 0.15 along its normal (2500 steps): it runs with positive
    temperatures; the incident shock meets the top boundary at the exact position g(t) (the top
    row's density crosses the mean of the jump within 3 cells of it); and along the wall the
    reflected front (the Mach stem) runs ahead of the point where the incident shock line would
    meet the wall, x_wall + 2 W t / sqrt(3), as in a Mach reflection."""
    w = W.dmr(Ms=6.0)
    steps = int(round(0.15 / w.meta["W"] / w.dt))
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    s.step(steps)
    rho, u, v, T = s.get_macro()
    assert _status(s) == 0
    assert T.min() > 0
    rho2 = w.meta["post"][0]
    t = steps * w.dt
    top = w.meta["segments"][1]
    g = top[1] + top[2] * t
    x = (np.arange(w.nx) + 0.5) * w.dx
    half = 0.5 * (rho2 + W.DMR_PRE[0])
    i_top = np.where(rho[-1] > half)[0].max()
    assert abs(x[i_top] - g) <= 3 * w.dx
    i_wall = np.where(rho[0] > half)[0].max()
    foot = w.meta["x_wall"] + 2.0 * w.meta["W"] * t / np.sqrt(3.0)
    assert x[i_wall] > foot + 5 * w.dx
