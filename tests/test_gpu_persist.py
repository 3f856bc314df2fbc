"""Persistent steps (variants 13 and 14): one cooperative launch runs all the steps of a call, the
CTAs meeting at a grid barrier between steps, with the tile bodies of variants 9 (ring-parallel
8 x 4) and 2 (32 x 16). Each node's arithmetic is theirs, so every result must be theirs bit for
bit: on every boundary kind, odd and even step counts, runs longer than one launch, a rejected
state, and the fall-back to one-step launches for a solve with boundary segments. The barrier's
bounded wait is tested on its own: without one CTA's arrival it must give up and report
FDLBM_E_TIMEOUT.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402

PAIRS = [(13, 9), (14, 2)]  # persistent variant, its one-step tile body


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    F.lib()


def _smooth(nx, ny, seed, amp=0.1, base=(1.0, 0.3, -0.2, 1.0)):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * (np.arange(nx) + 0.5) / nx
    y = 2 * np.pi * (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for b in base:
        a1, a2, p1, p2 = rng.uniform(-1, 1, 4)
        out.append(b + amp * (abs(b) + 0.5) * (a1 * np.sin(X + p1) + a2 * np.cos(Y + 2 * X + p2)))
    return out


def _padded(s, nx, ny):
    f = s.get_f_region(-2, -2, nx + 4, ny + 4)
    f[:, :2, :2] = f[:, :2, -2:] = f[:, -2:, :2] = f[:, -2:, -2:] = 0  # corners: never read
    return f


CASES = [
    (400, 4, (1, 1, 0, 0), 41),
    (37, 23, (0, 0, 0, 0), 40),
    (45, 19, (1, 2, 3, 1), 33),
    (130, 70, (2, 1, 1, 3), 20),
    (1, 6, (0, 0, 3, 2), 15),
    (4000, 4, (1, 1, 0, 0), 12),
]


@pytest.mark.parametrize("prec", [F.FDLBM_FP64, F.FDLBM_FP32_STORE])
@pytest.mark.parametrize("nx,ny,bc,steps", CASES)
def test_persistent_steps_equal_one_step_launches_bit_for_bit(prec, nx, ny, bc, steps):
    bstate = np.zeros((4, 4))
    for side in range(4):
        bstate[side] = (1.1 + 0.1 * side, 0.2, -0.1, 0.9)
    fields = _smooth(nx, ny, nx * 100 + ny)
    for vp, v1 in PAIRS:
        out = []
        for v in (v1, vp):
            s = F.Solver(nx, ny, 1e-3, 1.2e-3, 1e-5, 1.5e-5, 1.5, bc, prec, 0, bstate)
            s.set_variant(v)
            s.set_macro(*fields)
            s.step(steps)
            out.append(_padded(s, nx, ny))
            assert s.sync() == 0 and s.steps_done == steps
            s.close()
        assert np.array_equal(out[0], out[1]), (vp, v1)


def test_persistent_run_longer_than_one_launch():
    """5000 steps of a 400 x 4 Sod tube: two launches (4096 + 904 steps) against 5000 one-step
    launches, FP64, every bit of rho, u, v, T."""
    w = W.sod(nx=400, ny=4, steps=5000)
    res = []
    for v in (9, 13):
        s = F.Solver.from_workload(w, F.FDLBM_FP64)
        s.set_variant(v)
        s.step(w.steps)
        res.append(s.get_macro())
        s.close()
    for a, b in zip(*res):
        assert np.array_equal(a, b)


def test_persistent_run_reports_a_rejected_state():
    """Ms = 20 into gas at rest: rejected at its second step; a persistent call of 5 steps reports
    FDLBM_E_NUMERIC like the one-step launches."""
    w = W.shock_tube(nx=200, ny=4, steps=5, Ms=20.0, U=0.0, T1=1.0, lam=5.0)
    for v in (13, 14):
        s = F.Solver.from_workload(w, F.FDLBM_FP64)
        s.set_variant(v)
        s.step(5)
        with pytest.raises(F.FdlbmError) as ei:
            s.sync()
        assert ei.value.code == F.FDLBM_E_NUMERIC
        s.close()


def test_autotune_times_persistent_variants_without_advancing_the_state():
    w = W.sod(nx=400, ny=4, steps=10)
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    f0 = s.get_f()
    for trial_steps in (3, 40):  # on this grid every variant is timed over at least 32 steps
        times = s.autotune(trial_steps)
        assert times[13] > 0 and times[14] > 0
        assert np.array_equal(s.get_f(), f0) and s.steps_done == 0
        assert s.health() == 0


def test_solve_with_segments_takes_one_step_launches():
    w = W.dmr(Ms=6.0, nx=125, ny=50, dx=4e-3, dt=4e-5)
    out = []
    for v in (9, 13):
        s = F.Solver.from_workload(w, F.FDLBM_FP64)
        s.set_variant(v)
        s.step(60)
        out.append(_padded(s, w.nx, w.ny))
        assert s.sync() == 0
        s.close()
    assert np.array_equal(out[0], out[1])


def test_grid_barrier_gives_up_without_every_arrival():
    rc, done = F.fdlbm_selftest_grid_barrier(1, 3000)
    assert rc == F.FDLBM_E_TIMEOUT and done == 0
    rc, done = F.fdlbm_selftest_grid_barrier(0, 1 << 20, rounds=8)
    assert rc == F.FDLBM_OK and done == 1
