"""The double Mach reflection's set-up (Sec. 5.2.2, Eq. 27) and the oracle's moving boundary segments.

Pins:
- the workload's shock line and top-boundary split reproduce the paper's printed formulas
  h(x, t) = sqrt(3) (x - 80 dx) - 40 t and g(t) = 80 dx + (sqrt(3)/3)(0.2 + 40 t) at Ms = 20;
- a segment reduces to the plain side when it covers all of it or none of it (bit for bit);
- the ghosts follow the split at every step's time: f_eq of the segment's state below it, the
  side's own rule (Dirichlet state, wall mirror) beyond it.
"""
import math

import numpy as np
import pytest

from oracle import fdlbm as O
from paper_0801_4169_gb300 import workloads as W

Q = 33


def _sim(w, segments=None):
    s = O.Sim(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, w.bstate)
    for seg in (w.meta["segments"] if segments is None else segments):
        s.set_segment(*seg)
    s.set_macro(*w.macros())
    return s


def test_dmr_set_up_follows_the_papers_formulas():
    """At Ms = 20, dx = 1e-3 (500 x 200): post-shock state (400/67, 13.3 cos 30, -13.3 sin 30,
    89.2775) above y = sqrt(3)(x - 0.08), gas at rest (2, 0, 0, 0.5) below; the top split is
    g(t) = 0.08 + (0.2 + 40 t)/sqrt(3) and the bottom wall starts at x = 0.08."""
    w = W.dmr(Ms=20.0)
    post = w.meta["post"]
    assert post[0] == pytest.approx(400.0 / 67.0, rel=1e-12)
    assert math.hypot(post[1], post[2]) == pytest.approx(13.3, abs=1e-3)
    assert math.degrees(math.atan2(-post[2], post[1])) == pytest.approx(30.0, abs=1e-9)
    assert post[3] == pytest.approx(89.2775, abs=5e-5)
    x = (np.arange(w.nx) + 0.5) * w.dx
    y = (np.arange(w.ny) + 0.5) * w.dx
    X, Y = np.meshgrid(x, y)
    behind = Y >= math.sqrt(3.0) * (X - 80 * 1e-3) - 40.0 * 0.0
    assert np.array_equal(w.rho == post[0], behind)
    bottom, top = w.meta["segments"]
    assert bottom[:4] == (2, 0.08, 0.0, True)
    for t in (0.0, 1e-3, 7.5e-3):
        g = 80 * 1e-3 + math.sqrt(3.0) / 3.0 * (0.2 + 40.0 * t)
        assert top[1] + top[2] * t == pytest.approx(g, rel=1e-14)
    assert w.bc == (W.DIRICHLET, W.OUTFLOW, W.WALL, W.DIRICHLET)
    assert tuple(w.bstate[0]) == post and tuple(w.bstate[3]) == W.DMR_PRE


def test_segment_covering_all_or_nothing_is_the_plain_side():
    """A segment over the whole of a Dirichlet side with the side's own state, or over none of a
    wall side, leaves every value of a 20-step run bit for bit unchanged."""
    w = W.dmr(Ms=4.0, nx=40, ny=20, dx=4e-3, dt=4e-5)
    ref = _sim(w, segments=[])
    assert ref.step(20) == 0
    a = _sim(w, segments=[(3, 1e9, 0.0, True, tuple(w.bstate[3])), (2, -1e9, 0.0, True, w.meta["post"])])
    assert a.step(20) == 0
    assert np.array_equal(a.get_f_padded(), ref.get_f_padded())


def test_segment_ghosts_follow_the_split_in_time():
    """After k steps, the top ghost rows hold f_eq(post) at the columns with (i + 1/2) dx below
    g(k dt) and f_eq(pre) beyond; the bottom ghost rows hold f_eq(post) before x = 0.08 and the
    mirror of rows 0 and 1 from there on."""
    w = W.dmr(Ms=4.0, nx=40, ny=20, dx=4e-3, dt=4e-5)
    s = _sim(w)
    top = w.meta["segments"][1]
    fe_post = O.feq(*w.meta["post"])
    fe_pre = O.feq(*W.DMR_PRE)
    mirror = [0] + [1 + 8 * k + ((8 - (d + 1)) % 8 + 7) % 8 for k in range(4) for d in range(8)]
    seen = set()
    for k in (0, 7, 30):
        if k:
            assert s.step(k - s.steps_done) == 0
        fp = s.get_f_padded()  # [q][j + 2][i + 2]
        split = top[1] + top[2] * (k * w.dt)
        for i in range(w.nx):
            x = (i + 0.5) * w.dx
            for jj in (w.ny + 2, w.ny + 3):
                want = fe_post if x < split else fe_pre
                seen.add(x < split)
                assert np.array_equal(fp[:, jj, i + 2], want)
            for layer in (0, 1):  # ghost row -1 - layer mirrors row layer
                got = fp[:, 1 - layer, i + 2]
                if x < 0.08:
                    assert np.array_equal(got, fe_post)
                else:
                    assert np.array_equal(got, fp[mirror, 2 + layer, i + 2])
    assert seen == {True, False}


def test_dmr_reduced_runs_at_mach_6():
    """The paper's geometry on 125 x 50 (dx = 4e-3, dt = tau = 4e-5, lambda = 20) runs until the
    incident shock has moved 0.3 at Ms = 6; at Ms = 8 it is rejected within 50 steps (the scheme
    stops near Ms 6-7 into gas at rest, where the Eq. 27 data need Ms = 20)."""
    w = W.dmr(Ms=6.0, nx=125, ny=50, dx=4e-3, dt=4e-5)
    s = _sim(w)
    assert s.step(int(round(0.3 / w.meta["W"] / w.dt))) == 0
    rho, u, v, T = s.get_macro()
    assert T.min() > 0 and rho.max() > w.meta["post"][0]
    w8 = W.dmr(Ms=8.0, nx=125, ny=50, dx=4e-3, dt=4e-5)
    s8 = _sim(w8)
    assert s8.step(50) == -4
