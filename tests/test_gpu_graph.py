"""Graph-replayed steps (variant 15): the ring-parallel 8 x 4 step (variant 9) launched from CUDA
graphs of 32 steps, captured once per starting buffer on the solve's private stream; the steps of a
call beyond a multiple of 32 are launched one by one. The kernels and their arguments are those of
variant 9, so every result must be its result bit for bit: on every boundary kind, over calls whose
step counts leave remainders of either parity, on the legacy and on a caller's stream, from either
buffer, for a rejected state, and for the precisions and solves (boundary segments) that launch the
steps one by one.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402

GRAPH, ONE_BY_ONE = 15, 9


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
    (400, 4, (1, 1, 0, 0)),
    (37, 23, (0, 0, 0, 0)),
    (45, 19, (1, 2, 3, 1)),
    (130, 70, (2, 1, 1, 3)),
]
CALLS = (5, 64, 33, 100)  # 0, 2, 1 and 3 replays, then 5, 0, 1 and 4 single launches


@pytest.mark.parametrize("prec", [F.FDLBM_FP64, F.FDLBM_FP32_STORE])
@pytest.mark.parametrize("nx,ny,bc", CASES)
def test_graph_replayed_steps_equal_one_by_one_launches(prec, nx, ny, bc):
    bstate = np.zeros((4, 4))
    for side in range(4):
        bstate[side] = (1.1 + 0.1 * side, 0.2, -0.1, 0.9)
    fields = _smooth(nx, ny, nx * 31 + ny)
    runs = []
    for v in (ONE_BY_ONE, GRAPH):
        s = F.Solver(nx, ny, 1e-3, 1.2e-3, 1e-5, 1.5e-5, 1.5, bc, prec, 0, bstate)
        s.set_variant(v)
        s.set_macro(*fields)
        states = []
        for n in CALLS:
            s.step(n)
            states.append(_padded(s, nx, ny))
        assert s.sync() == 0 and s.steps_done == sum(CALLS)
        s.close()
        runs.append(states)
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_graph_replayed_steps_on_a_callers_stream():
    w = W.sod(nx=400, ny=4)
    out = []
    for v in (ONE_BY_ONE, GRAPH):
        st = torch.cuda.Stream()
        s = F.Solver.from_workload(w, F.FDLBM_FP64, stream=st)
        s.set_variant(v)
        s.step(96)
        s.step(37)
        out.append(s.get_f())
        assert s.sync() == 0
        s.close()
    assert np.array_equal(out[0], out[1])


def test_graph_replayed_steps_from_the_second_buffer():
    """An odd step count leaves the state in the second buffer; the graph that starts from that
    buffer takes over, and the one from the first after another odd count."""
    w = W.riemann4q(n=64, steps=10)
    out = []
    for v in (ONE_BY_ONE, GRAPH):
        s = F.Solver.from_workload(w, F.FDLBM_FP32_STORE)
        s.set_variant(v)
        s.step(7)
        assert F.fdlbm_current_buffer(s.h) == 1
        s.step(64)
        s.step(35)
        assert F.fdlbm_current_buffer(s.h) == 0
        s.step(32)
        out.append(s.get_f())
        assert s.sync() == 0 and s.steps_done == 7 + 64 + 35 + 32
        s.close()
    assert np.array_equal(out[0], out[1])


def test_rejected_state_inside_a_graph_replay_is_reported():
    """Shock Mach 20 into gas at rest fails at its second step: a call of 64 steps (two replays)
    reports FDLBM_E_NUMERIC, and the error stays until set_macro."""
    w = W.shock_tube(nx=200, ny=4, steps=2, Ms=20.0, U=0.0, T1=1.0, lam=5.0)
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    s.set_variant(GRAPH)
    s.step(64)
    with pytest.raises(F.FdlbmError) as ei:
        s.sync()
    assert ei.value.code == F.FDLBM_E_NUMERIC
    with pytest.raises(F.FdlbmError):
        s.step(32)
    s.set_macro(*W.sod(nx=200, ny=4).macros())
    s.step(40)
    assert s.sync() == 0
    s.close()


@pytest.mark.parametrize("prec", [F.FDLBM_FP32_STORE_DW, F.FDLBM_FNEQ32])
def test_other_precisions_launch_the_steps_one_by_one(prec):
    w = W.riemann4q(n=64, steps=10)
    out = []
    for v in (ONE_BY_ONE, GRAPH):
        s = F.Solver.from_workload(w, prec)
        s.set_variant(v)
        s.step(70)
        out.append(s.get_f())
        assert s.sync() == 0
        s.close()
    assert np.array_equal(out[0], out[1])


def test_solve_with_segments_launches_the_steps_one_by_one():
    w = W.dmr(Ms=6.0, nx=125, ny=50, dx=4e-3, dt=4e-5)
    out = []
    for v in (ONE_BY_ONE, GRAPH):
        s = F.Solver.from_workload(w, F.FDLBM_FP64)
        s.set_variant(v)
        s.step(70)
        out.append(_padded(s, w.nx, w.ny))
        assert s.sync() == 0
        s.close()
    assert np.array_equal(out[0], out[1])
