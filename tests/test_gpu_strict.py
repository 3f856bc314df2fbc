"""FDLBM_FP64_STRICT on the GPU against the FP64 CPU oracle: bit for bit.

The strict path forms every value of Eqs. 3-5, 10-13 and 17 one IEEE FP64 operation at a time in
one fixed order, with no fused multiply-add (the order is written out at the top of
csrc/fdlbm_strict.cu). The oracle is plain C compiled without contraction, taking the operations
of the same equations in the paper's order. Where the two orders agree, so must every bit: these
tests compare the 64-bit patterns of f (interior and the ghost cross the stencil reads), of the
moments, and the step at which a state is rejected. Corners of the ghost ring are never read and
are left out.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fdlbm as O  # noqa: E402
from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402

STRICT = F.FDLBM_FP64_STRICT


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


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _cross(fp):
    """The padded buffer [q][j + 2][i + 2] without its four 2 x 2 corners."""
    out = fp.copy()
    out[:, :2, :2] = 0.0
    out[:, :2, -2:] = 0.0
    out[:, -2:, :2] = 0.0
    out[:, -2:, -2:] = 0.0
    return out


def _gpu_padded(s, nx, ny):
    return s.get_f_region(-2, -2, nx + 4, ny + 4)


def _status(s):
    try:
        return s.sync()
    except F.FdlbmError as e:
        return e.code


def _assert_same_bits(got, ref, what):
    bad = np.nonzero(_bits(got) != _bits(ref))
    assert bad[0].size == 0, "%s: %d values differ, first at %s: %r vs %r" % (
        what, bad[0].size, tuple(int(b[0]) for b in bad), got[tuple(b[0] for b in bad)], ref[tuple(b[0] for b in bad)])


CASES = [
    # nx, ny, bc, steps: every boundary kind, ragged blocks, a one-column grid
    (37, 23, (0, 0, 0, 0), 40),
    (45, 19, (1, 2, 3, 1), 40),
    (33, 9, (3, 3, 0, 0), 40),
    (70, 37, (2, 1, 1, 3), 30),
    (5, 3, (0, 0, 0, 0), 20),
    (1, 6, (0, 0, 3, 2), 20),
]


@pytest.mark.parametrize("nx,ny,bc,steps", CASES)
def test_strict_f_and_moments_equal_the_oracle_bit_for_bit(nx, ny, bc, steps):
    bstate = np.zeros((4, 4))
    for side in range(4):
        bstate[side] = (1.1 + 0.1 * side, 0.2, -0.1, 0.9)
    fields = _smooth(nx, ny, nx * 100 + ny)
    s = F.Solver(nx, ny, 1e-3, 1.2e-3, 1e-5, 1.5e-5, 1.5, bc, STRICT, 0, bstate)
    s.set_macro(*fields)
    o = O.Sim(nx, ny, 1e-3, 1.2e-3, 1e-5, 1.5e-5, 1.5, bc, bstate)
    o.set_macro(*fields)
    # the initial condition (Eq. 10 at every node, Dirichlet ghosts) already agrees
    _assert_same_bits(_cross(_gpu_padded(s, nx, ny)), _cross(o.get_f_padded()), "f at t = 0")
    s.step(steps)
    assert o.step(steps) == 0
    _assert_same_bits(_cross(_gpu_padded(s, nx, ny)), _cross(o.get_f_padded()), "f")
    for got, ref, name in zip(s.get_macro(), o.get_macro(), ("rho", "u", "v", "T")):
        _assert_same_bits(got, ref, name)


@pytest.mark.parametrize("flags", [O.NO_LW, O.NO_DISP, O.NO_VISC, O.SWITCH_CONST, O.NO_LW | O.NO_DISP | O.NO_VISC])
def test_strict_scheme_variants_equal_the_oracle_bit_for_bit(flags):
    """The Sec. 4 variants of Eq. 17 (lines II, III or IV dropped; the switch held at lambda)."""
    nx, ny = 24, 16
    fields = _smooth(nx, ny, 5, amp=0.2)
    s = F.Solver(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 0.8, (0, 0, 0, 0), STRICT, flags)
    s.set_macro(*fields)
    s.step(25)
    o = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 0.8, (0, 0, 0, 0), flags=flags)
    o.set_macro(*fields)
    assert o.step(25) == 0
    _assert_same_bits(_cross(_gpu_padded(s, nx, ny)), _cross(o.get_f_padded()), "f")


def test_strict_sod_and_riemann_suite_equal_the_oracle_bit_for_bit():
    """The Sec. 5.1 tubes at the paper's parameters (400 x 1 here, outflow ends) over 500 steps."""
    for name in ("sod", "lax", "sjogreen", "collision"):
        w = W.riemann1d(name, nx=400) if name != "sod" else W.sod(nx=400, ny=1)
        s = F.Solver.from_workload(w, STRICT)
        s.step(500)
        o = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
        o.set_macro(*w.macros())
        assert o.step(500) == 0
        for got, ref, fld in zip(s.get_macro(), o.get_macro(), ("rho", "u", "v", "T")):
            _assert_same_bits(got, ref, "%s %s" % (name, fld))


def test_strict_double_mach_segments_equal_the_oracle_bit_for_bit():
    """Reduced double Mach reflection (125 x 50, Ms = 6): the top boundary's moving Dirichlet
    segment and the bottom's Dirichlet stretch before the wall, applied with each new state's time."""
    w = W.dmr(Ms=6.0, nx=125, ny=50, dx=4e-3, dt=4e-5)
    s = F.Solver.from_workload(w, STRICT)
    s.step(150)
    assert _status(s) == 0
    o = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
    for seg in w.meta["segments"]:
        o.set_segment(*seg)
    o.set_macro(*w.macros())
    assert o.step(150) == 0
    _assert_same_bits(_cross(_gpu_padded(s, w.nx, w.ny)), _cross(o.get_f_padded()), "f")


@pytest.mark.parametrize("flags", [0, O.NO_DISP])
def test_strict_fig3_tube_equals_the_oracle_bit_for_bit(flags):
    """The Sec. 4 Fig. 3 tube (kappa = 1.7e4, two shocks), 3000 steps, with and without line III:
    every bit of rho, u, v, T. The FP64 fast path is held to the oracle's rounding spread on this
    run (its shocks amplify rounding-order differences); the strict path has no spread to hide in."""
    w = W.riemann1d("fig3", nx=400)
    s = F.Solver(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, STRICT, flags, w.bstate)
    s.set_macro(*w.macros())
    s.step(w.steps)
    o = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate, flags=flags)
    o.set_macro(*w.macros())
    assert o.step(w.steps) == 0
    for got, ref, fld in zip(s.get_macro(), o.get_macro(), ("rho", "u", "v", "T")):
        _assert_same_bits(got, ref, fld)


def test_strict_reflection_downscale_equals_the_oracle_bit_for_bit():
    """The regular reflection (Sec. 5.2.1) on its 300 x 75 downscale (kappa = 7.4e6 in the top state, walls, Dirichlet
    and outflow sides), 400 steps: every f of the interior and the ghost cross."""
    w = W.reflection(nx=300, ny=75)
    s = F.Solver.from_workload(w, STRICT)
    s.step(400)
    assert _status(s) == 0
    o = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
    o.set_macro(*w.macros())
    assert o.step(400) == 0
    _assert_same_bits(_cross(_gpu_padded(s, w.nx, w.ny)), _cross(o.get_f_padded()), "f")


def _fail_step_pair(w, max_steps):
    """Step the strict GPU path and the oracle one step at a time; f agrees bit for bit before each
    step. Returns the 1-based index of the step each side rejects (0: none within max_steps)."""
    s = F.Solver.from_workload(w, STRICT)
    o = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
    o.set_macro(*w.macros())
    kg = ko = 0
    for k in range(1, max_steps + 1):
        _assert_same_bits(_cross(_gpu_padded(s, w.nx, w.ny)), _cross(o.get_f_padded()), "f before step %d" % k)
        s.step(1)
        g_bad = _status(s) == F.FDLBM_E_NUMERIC
        o_bad = o.step(1) != 0
        kg = kg or (k if g_bad else 0)
        ko = ko or (k if o_bad else 0)
        if g_bad or o_bad:
            break
    return kg, ko


@pytest.mark.parametrize("seed,expect", [(0, 2), (1, 3), (2, 4)])
def test_strict_rejects_the_posed_four_quadrant_states_at_the_oracles_step(seed, expect):
    """The four-quadrant states as first posed (rho in [0.1, 2], p in [0.03, 1.5], Mach <= 10,
    lambda = 1; 48 x 48 at the 4096^2 spacing): both sides reject the same step."""
    w = W.riemann4q(n=48, seed=seed, lam=1.0, mach_max=10.0, rho_range=(0.1, 2.0), p_range=(0.03, 1.5))
    assert _fail_step_pair(w, 10) == (expect, expect)


def test_strict_rejects_mach20_into_rest_at_the_oracles_step():
    """Shock Mach 20 into gas at rest (the strong tube as first posed) and the Colella problem
    (Eq. 24): rejected at the same step on both sides, with equal bits up to it."""
    w = W.shock_tube(nx=200, ny=4, steps=2, Ms=20.0, U=0.0, T1=1.0, lam=5.0)
    kg, ko = _fail_step_pair(w, 5)
    assert kg == ko and kg > 0
    kg, ko = _fail_step_pair(W.riemann1d("colella", nx=200), 5)
    assert kg == ko and kg > 0


def test_strict_agrees_with_the_fp64_path_to_rounding():
    """FDLBM_FP64 (FMA contraction, its own summation trees and Newton reciprocals) against the
    strict path on a smooth flow after 200 steps: within 1e-12 of max|f|, and not bit for bit."""
    nx, ny = 64, 48
    fields = _smooth(nx, ny, 11)
    out = {}
    for prec in (F.FDLBM_FP64, STRICT):
        s = F.Solver(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 1.0, (0, 0, 0, 0), prec)
        s.set_macro(*fields)
        s.step(200)
        out[prec] = s.get_f()
    a, b = out[F.FDLBM_FP64], out[STRICT]
    assert np.max(np.abs(a - b)) <= 1e-12 * np.abs(b).max()
    assert not np.array_equal(a, b)


def test_strict_checkpoint_and_variants(tmp_path):
    """Checkpoint and resume are bitwise; set_variant is accepted and changes nothing; autotune
    times nothing; batches and the no-alloc step refuse the strict precision."""
    w = W.riemann4q(n=40, steps=10)
    a = F.Solver.from_workload(w, STRICT)
    a.step(5)
    path = str(tmp_path / "strict.ck")
    F.fdlbm_save(a.h, path)
    a.step(5)
    fa = a.get_f()
    b = F.Solver.from_workload(w, STRICT)
    F.fdlbm_load(b.h, path)
    F.fdlbm_set_variant(b.h, 2)
    b.step(5)
    assert np.array_equal(fa, b.get_f())
    times = b.autotune(2)
    assert all(t == 0 for t in times)
    bt = F.fdlbm_batch_create()
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_batch_add(bt, b.h)
    assert ei.value.code == F.FDLBM_E_ARG
    F.fdlbm_batch_destroy(bt)
