"""Which posed problems the scheme rejects, and whether the rejection is the scheme's or FP64's.

Several problems fail within a few steps in the FP64 oracle: a node reaches T <= 0 (or n <= 0),
where Eq. 16 is undefined. At these states the equilibrium of Eq. 10 is badly conditioned
(kappa = sum |f_eq| / n up to 1e12), so an FP64 rounding could in principle cause the failure.
The extended-precision restatement (oracle/fdlbm_mp.py, 40 digits) settles it: when the same node
reaches T <= 0 at 40 digits, and 40 and 60 digits agree, the scheme itself (under this build's
readings) produces that state, and FP64 only reproduces it.

Failures are searched with the FP64 oracle; the decisive node is then recomputed at 40 digits on
the whole grid (1-D problems) or on a window around it. A window keeps the domain's boundary kind
on the sides it shares with the domain and takes outflow elsewhere; it is wide enough (3 nodes per
step plus 3) that the node's value is bit for bit the full domain's in FP64, which the test checks.
"""
from dataclasses import replace

import mpmath as mp
import numpy as np
import pytest

from oracle import fdlbm as O
from oracle import fdlbm_mp as M
from paper_0801_4169_gb300 import workloads as W

OUT = O.OUTFLOW


def _sim(w):
    s = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
    s.set_macro(*w.macros())
    return s


def _mp(w, dps=40):
    s = M.MPSim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate, dps=dps)
    s.set_macro(*w.macros())
    return s


def _fail_step(w, max_steps):
    """The 1-based index of the FP64 step that rejects its input, or 0 if max_steps all ran."""
    s = _sim(w)
    for k in range(1, max_steps + 1):
        if s.step(1):
            return k
    return 0


def _worst_after(w, steps):
    """FP64 macros after `steps` steps and the (j, i) of the lowest temperature."""
    s = _sim(w)
    assert s.step(steps) == 0
    m = s.get_macro()
    T = np.where(np.isfinite(m[3]), m[3], -np.inf)
    j, i = np.unravel_index(np.argmin(T), T.shape)
    return m, int(j), int(i)


def _window(w, j0, i0, R):
    ja, jb = max(0, j0 - R), min(w.ny, j0 + R + 1)
    ia, ib = max(0, i0 - R), min(w.nx, i0 + R + 1)
    bc = (w.bc[0] if ia == 0 else OUT, w.bc[1] if ib == w.nx else OUT,
          w.bc[2] if ja == 0 else OUT, w.bc[3] if jb == w.ny else OUT)
    sub = replace(w, nx=ib - ia, ny=jb - ja, bc=bc,
                  rho=w.rho[ja:jb, ia:ib].copy(), u=w.u[ja:jb, ia:ib].copy(),
                  v=w.v[ja:jb, ia:ib].copy(), T=w.T[ja:jb, ia:ib].copy())
    return sub, j0 - ja, i0 - ia


def _decide(w, steps, dps=40):
    """T at the worst FP64 node after `steps` steps: (FP64 value, value at dps digits)."""
    m, j, i = _worst_after(w, steps)
    sub, jj, ii = _window(w, j, i, 3 * steps + 3)
    s = _sim(sub)
    assert s.step(steps) == 0
    assert s.get_macro()[3][jj, ii] == m[3][j, i]  # the window reproduces the node bit for bit
    t = _mp(sub, dps)
    assert t.step(steps) == 0
    return m[3][j, i], t.macros()[3][jj, ii]


# ---------------------------------------------------------------------------------------------
# the restatement itself


def test_mp_restatement_matches_the_fp64_oracle_where_fp64_is_well_conditioned():
    """Two independent readings of Eqs. 1-17 (C in FP64, mpmath at 40 digits) agree to FP64
    rounding on a Sod tube and on a 2-D four-quadrant problem (kappa ~ 1), every boundary kind
    used by the problems below included (outflow, periodic, Dirichlet, wall)."""
    cases = [(W.sod(nx=16, ny=1), 4), (W.riemann4q(n=8, seed=0), 3)]
    refl = W.reflection(nx=10, ny=6)
    refl = replace(refl, rho=np.full((6, 10), 1.0), u=np.full((6, 10), 0.5), v=np.full((6, 10), 0.1),
                   T=np.full((6, 10), 1.0), bstate=np.array([[1.2, 0.3, 0.0, 0.9], [0] * 4, [0] * 4,
                                                             [0.8, 0.0, -0.2, 1.1]]))
    cases.append((refl, 3))
    for w, steps in cases:
        o = _sim(w)
        assert o.step(steps) == 0
        t = _mp(w)
        assert t.step(steps) == 0
        for a, b in zip(o.get_macro(), t.macros()):
            b = np.array([[float(x) for x in row] for row in b])
            assert np.max(np.abs(a - b)) <= 5e-14 * max(1.0, np.max(np.abs(b)))


def test_forty_digits_are_enough_at_the_worst_states():
    """At the Colella state (kappa ~ 2e12) 40 and 60 digits agree to 1e-25 after one step, so the
    40-digit results below are exact for the purpose of deciding a sign."""
    w = W.riemann1d("colella", nx=16)
    a, b = _mp(w, 40), _mp(w, 60)
    a.step(1)
    b.step(1)
    with mp.workdps(60):
        for x, y in zip(a.macros()[3][0], b.macros()[3][0]):
            assert abs(x - y) <= mp.mpf("1e-25") * abs(y)


# ---------------------------------------------------------------------------------------------
# 1-D problems: the whole grid at 40 digits


def _decide_1d(w):
    o = _sim(w)
    assert o.step(1) == 0
    T64 = o.get_macro()[3][0]
    t = _mp(w)
    assert t.step(1) == 0
    Tmp = t.macros()[3][0]
    i = int(np.argmin(T64))
    return T64[i], Tmp[i], min(Tmp), o.step(1), t.step(1)


@pytest.mark.parametrize("lam", [1.0, 20.0])
def test_mach20_into_rest_fails_in_exact_arithmetic(lam):
    """Shock Mach 20 into gas at rest (1, 0, 0, 1), the strong-tube problem as first posed:
    one step makes the first cold node's temperature -22.70 at 40 digits as in FP64 (the two agree
    to 1e-9), so the second step rejects it in both. The scheme, not FP64, fails here."""
    w = W.shock_tube(nx=24, ny=1, steps=2, Ms=20.0, U=0.0, T1=1.0, lam=lam, x0_frac=0.5)
    T64, Tmp, Tmin, rc64, rcmp = _decide_1d(w)
    assert Tmp < -20.0 and T64 < -20.0
    assert abs(T64 - float(Tmp)) <= 1e-9 * abs(float(Tmp))
    assert rc64 == -4 and rcmp == -4


@pytest.mark.parametrize("lam", [1.0, 20.0])
def test_dmr_normal_shock_fails_in_exact_arithmetic(lam):
    """Sec. 5.2.2, Eq. 27: the normal shock behind the double Mach reflection, (400/67, 13.3, 0,
    89.2775) into (2, 0, 0, 0.5) at rest, normal Mach 20. Its first cold node reaches T < 0 after
    one step at 40 digits as in FP64: the scheme rejects the Eq. 27 data."""
    w = W.shock_tube(nx=24, ny=1, steps=2, Ms=20.0, U=0.0, T1=0.5, rho1=2.0, lam=lam, x0_frac=0.5)
    assert w.meta["post"][0] == pytest.approx(400.0 / 67.0, rel=1e-12)
    T64, Tmp, Tmin, rc64, rcmp = _decide_1d(w)
    assert Tmp < 0 and T64 < 0
    assert abs(T64 - float(Tmp)) <= 1e-8 * abs(float(Tmp))
    assert rc64 == -4 and rcmp == -4


def test_colella_fails_in_exact_arithmetic():
    """Sec. 5.1, Eq. 24 (T = 1000 | 0.01, lambda = 20): the first cold node reaches T = -0.0261 after
    one step at 40 digits. FP64 gives -0.0261 too, off in the 6th digit (kappa ~ 2e12), but the sign
    is the scheme's."""
    w = W.riemann1d("colella", nx=24)
    T64, Tmp, Tmin, rc64, rcmp = _decide_1d(w)
    assert float(Tmp) == pytest.approx(-0.02605035, rel=1e-6)
    assert abs(T64 - float(Tmp)) <= 1e-4 * abs(float(Tmp))
    assert rc64 == -4 and rcmp == -4


# ---------------------------------------------------------------------------------------------
# 2-D problems: FP64 scans, then the decisive node at 40 digits on a window


def _c5(seed, lam):
    """The four-quadrant states as first posed: rho in [0.1, 2], p in [0.03, 1.5], local Mach <= 10;
    the scan grid is 48 x 48 at the 4096^2 problem's spacing (dx = 2.5e-4, dt = tau = 2.5e-6)."""
    return W.riemann4q(n=48, seed=seed, lam=lam, mach_max=10.0, rho_range=(0.1, 2.0), p_range=(0.03, 1.5))


@pytest.mark.parametrize("lam,expect", [(1.0, (2, 3, 4)), (3.0, (2, 5, 0)), (20.0, (2, 9, 0))])
def test_four_quadrant_posed_ranges_scan(lam, expect):
    """The FP64 oracle on those ranges, seeds 0-2: at lambda = 1 every seed is rejected within 4 steps; from lambda = 3 to 20 seed 2 runs 2000 steps while
    seeds 0 and 1 are rejected within 9. (0 = all 2000 steps ran.)"""
    got = tuple(_fail_step(_c5(seed, lam), 2000 if e == 0 else 20) for seed, e in enumerate(expect))
    assert got == expect


@pytest.mark.parametrize("seed,lam,steps", [(0, 1.0, 1), (1, 1.0, 2)])
def test_four_quadrant_posed_failures_hold_in_exact_arithmetic(seed, lam, steps):
    """The node that fails first (a quadrant interface) has T < 0 at 40 digits too, agreeing with
    FP64 to 1e-6: these ranges are rejected by the scheme."""
    T64, Tmp = _decide(_c5(seed, lam), steps)
    assert Tmp < 0 and T64 < 0
    assert abs(T64 - float(Tmp)) <= 1e-6 * abs(float(Tmp))


def test_reflection_sharp_shock_needs_strong_viscosity():
    """The regular reflection (Sec. 5.2.1, Eq. 26) on the 300 x 75 downscale (dx = 4e-3, dt = tau = 1e-5), started from a sharp
    30-degree incident shock through the top-left corner: rejected within 4 steps at lambda = 1 and 5,
    while at lambda = 20, the value the 1200 x 300 run uses, it runs (200 steps here; 4000 in a longer scan)."""
    for lam, lo, hi in ((1.0, 1, 5), (5.0, 1, 5)):
        k = _fail_step(W.reflection(nx=300, ny=75, init="shock", lam=lam), 10)
        assert lo <= k <= hi
    assert _fail_step(W.reflection(nx=300, ny=75, init="shock", lam=20.0), 200) == 0


def test_reflection_sharp_shock_failure_holds_in_exact_arithmetic():
    """At lambda = 1 the first bad node (next to the wall, behind the incident shock) has T < 0 after
    3 steps at 40 digits too; FP64 is off by 4e-6 relative there (kappa ~ 7e6 in the top state)."""
    T64, Tmp = _decide(W.reflection(nx=300, ny=75, init="shock", lam=1.0), 3)
    assert Tmp < 0 and T64 < 0
    assert abs(T64 - float(Tmp)) <= 2e-5 * abs(float(Tmp))


def test_reflection_time_step_1e5_at_dx_1e3_fails():
    """dt = 1e-5 at dx = 1e-3 (kappa_x = 0.2 in the Mach-20 stream), the pair first posed for it, on a 120 x 40
    window of the reflection at that spacing: rejected within 100 steps from the post-shock start
    (lambda 1 and 20) and within 2 from the sharp shock. With dt = tau = 2.5e-6 the same problem
    runs the same physical time (400 steps)."""
    for init, lam, limit in (("post", 1.0, 100), ("post", 20.0, 100), ("shock", 20.0, 2)):
        w = W.reflection(nx=120, ny=40, dx=1e-3, dt=1e-5, lam=lam, init=init, height=0.04)
        assert 1 <= _fail_step(w, limit) <= limit
    w = W.reflection(nx=120, ny=40, dx=1e-3, dt=2.5e-6, lam=20.0, init="post", height=0.04)
    assert _fail_step(w, 400) == 0


def test_strong_shocks_need_a_counter_stream_and_stop_near_mach_12():
    """Why the serving stream draws Ms from [2, 10] with the upstream at -(Ms - 2) c1 (FP64 oracle,
    600 x 1, dx = 1e-3, dt = tau = 1e-5, lambda = 2): Mach 10 runs 2000 steps with the upstream
    at -8 c1; Mach 15 and 25 are rejected within 100 steps even with the upstream at -0.9 Ms c1."""
    def fails_within(Ms, U, steps):
        return _fail_step(W.shock_tube(nx=600, ny=1, steps=steps, Ms=Ms, U=U), steps)
    assert fails_within(10.0, 8.0, 2000) == 0
    for Ms in (15.0, 25.0):
        assert 1 <= fails_within(Ms, 0.9 * Ms, 100) <= 100
