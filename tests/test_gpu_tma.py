"""The FP32-storage step whose tile arrives in shared memory by one tensor copy (variant 12).

Its node arithmetic is that of the other FP32-storage variants, so it must agree with them bit for
bit: on ragged grids with every boundary kind, on grids smaller than one 36 x 12 box (which run
the plain 32 x 8 tile), with both equilibria (FP64 and double word), through the handle and the
no-allocation entry point. The bounded wait that guards the copy is tested on its own: with no
arrival it must give up and report FDLBM_E_TIMEOUT, with one it must complete.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402

TMA = 12


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


CASES = [
    (37, 23, (0, 0, 0, 0), 40),
    (45, 19, (1, 2, 3, 1), 40),
    (33, 9, (3, 3, 0, 0), 40),
    (70, 37, (2, 1, 1, 3), 30),
    (130, 70, (1, 1, 3, 2), 30),
    (5, 3, (0, 0, 0, 0), 20),     # smaller than one box: the 32 x 8 tile runs
    (1, 6, (0, 0, 3, 2), 20),
]


@pytest.mark.parametrize("prec", [F.FDLBM_FP32_STORE, F.FDLBM_FP32_STORE_DW])
@pytest.mark.parametrize("nx,ny,bc,steps", CASES)
def test_tensor_copy_step_equals_the_other_tiles_bit_for_bit(prec, nx, ny, bc, steps):
    bstate = np.zeros((4, 4))
    for side in range(4):
        bstate[side] = (1.1 + 0.1 * side, 0.2, -0.1, 0.9)
    fields = _smooth(nx, ny, nx * 100 + ny)
    out = []
    for v in (1, TMA):
        s = F.Solver(nx, ny, 1e-3, 1.2e-3, 1e-5, 1.5e-5, 1.5, bc, prec, 0, bstate)
        s.set_variant(v)
        s.set_macro(*fields)
        s.step(steps)
        out.append(s.get_f_region(-2, -2, nx + 4, ny + 4))
        assert s.sync() == 0
        s.close()
    a, b = out
    for f in (a, b):  # ghost corners are never written or read
        f[:, :2, :2] = f[:, :2, -2:] = f[:, -2:, :2] = f[:, -2:, -2:] = 0
    assert np.array_equal(a, b)


def test_tensor_copy_step_at_the_full_four_quadrant_size():
    """4096^2, 20 steps, both equilibria: the tensor-copy tile against the staged 32 x 8 tile."""
    w = W.riemann4q(n=4096, steps=20)
    for prec in (F.FDLBM_FP32_STORE, F.FDLBM_FP32_STORE_DW):
        rho = []
        for v in (6, TMA):
            s = F.Solver.from_workload(w, prec)
            s.set_variant(v)
            s.step(w.steps)
            rho.append(s.get_macro()[0])
            assert s.sync() == 0
            s.close()
        assert np.array_equal(rho[0], rho[1])


def test_double_word_default_is_the_tensor_copy_tile():
    s = F.Solver.from_workload(W.riemann4q(n=96, steps=5), F.FDLBM_FP32_STORE_DW)
    assert F.fdlbm_get_variant(s.h) == TMA


def test_bounded_wait_gives_up_without_an_arrival():
    rc, done = F.fdlbm_selftest_wait(0, 2000)
    assert rc == F.FDLBM_E_TIMEOUT and done == 0
    rc, done = F.fdlbm_selftest_wait(1, 2000)
    assert rc == F.FDLBM_OK and done == 1
