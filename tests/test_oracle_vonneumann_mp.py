"""Pins of the oracle's high-precision von Neumann matrix (Sec. 4, Eqs. 18-20, mpmath).

- At zero wave number the stencil symbols vanish and G = (1 - dt/tau) I + (dt/tau) J. The moments
  of f^eq(n, u, T) reproduce (n, u, T) exactly (the constraints Eq. 10 is built on). So
  J = d f^eq / d f is a rank-4 projector and the spectrum is exactly {1 (x4), 1 - dt/tau (x29)},
  at any Mach number. A dropped or wrong term of Eq. 20 or Eq. 10 breaks this.
- The high-precision G equals the FP64 oracle's G, which the linearised-step test pins
  element by element, where that one is well conditioned.
- x <-> y symmetry of the velocity set.
- The sensitivity that makes the high precision necessary is shown explicitly.
"""
import mpmath as mp
import numpy as np
import pytest

from oracle import fdlbm as O
from oracle import vonneumann as V

DPS = 40


def _c(z):
    return complex(z)


def _match(a, b):
    """Max distance between two multisets of complex numbers, matched greedily."""
    a = list(a)
    err = 0.0
    for z in b:
        j = int(np.argmin([abs(z - w) for w in a]))
        err = max(err, abs(z - a[j]))
        a.pop(j)
    return err


@pytest.mark.parametrize("state,dt,tau", [((2.0, 30.0, 0.0, 1.0), 1e-5, 1e-5), ((1.0, 0.5, -0.3, 0.8), 1e-5, 1e-4),
                                          ((50.0 / 17.0, 16.7, -5.71578, 22.61), 1e-5, 2e-5)])
def test_zero_wavenumber_spectrum_is_that_of_a_projector(state, dt, tau):
    G = V.amplification_matrix_mp(state, 0.0, 0.0, 3e-3, 3e-3, dt, tau, 0.5, dps=DPS)
    ev = V.eigvals_mp(G, DPS)
    with mp.workdps(DPS):
        r = mp.mpf(dt) / mp.mpf(tau)
        near1 = [z for z in ev if abs(z - 1) < mp.mpf("1e-20")]
        rest = [z for z in ev if abs(z - 1) >= mp.mpf("1e-20")]
        assert len(near1) == 4 and len(rest) == 29
        assert max(abs(z - 1) for z in near1) < mp.mpf("1e-25")
        assert max(abs(z - (1 - r)) for z in rest) < mp.mpf("1e-25")


def test_mp_feq_is_the_c_oracle_feq():
    for st in [(1.0, 0.3, -0.2, 1.0), (2.0, 30.0, 0.0, 1.0), (50.0 / 17.0, 16.7, -5.71578, 22.61)]:
        a = np.array([float(x) for x in V.feq_mp(*st, dps=DPS)])
        b = O.feq(*st)
        assert np.max(np.abs(a - b)) <= 1e-14 * np.abs(b).sum()


@pytest.mark.parametrize("xi", [(0.3, 0.0), (2.0, -0.4), (np.pi, 1.1)])
def test_mp_matrix_equals_fp64_oracle_matrix_where_well_conditioned(xi):
    st = (1.0, 0.3, -0.2, 1.0)
    args = (3e-3, 2e-3, 1e-5, 2e-5, 0.5)
    Gm = V.amplification_matrix_mp(st, xi[0], xi[1], *args, dps=DPS)
    Gm = np.array([[_c(Gm[i, j]) for j in range(33)] for i in range(33)])
    Gd = V.amplification_matrix(st, xi[0], xi[1], *args)
    assert np.max(np.abs(Gm - Gd)) <= 1e-10 * np.abs(Gd).max()
    ev_m = [_c(z) for z in V.eigvals_mp(V.amplification_matrix_mp(st, xi[0], xi[1], *args, dps=DPS), DPS)]
    assert _match(ev_m, np.linalg.eigvals(Gd)) <= 1e-9


def test_x_and_y_are_equivalent():
    """Rotating the state and the wave vector by 90 degrees maps the velocity set onto itself."""
    a = V.eigvals_mp(V.amplification_matrix_mp((1.0, 3.0, 0.0, 1.0), 0.7, 0.0, 2e-3, 2e-3, 1e-5, 1e-5, 1.0,
                                               dps=DPS), DPS)
    b = V.eigvals_mp(V.amplification_matrix_mp((1.0, 0.0, 3.0, 1.0), 0.0, 0.7, 2e-3, 2e-3, 1e-5, 1e-5, 1.0,
                                               dps=DPS), DPS)
    with mp.workdps(DPS):
        rest = list(b)
        for z in a:
            j = min(range(len(rest)), key=lambda k: abs(z - rest[k]))
            assert abs(z - rest[j]) < mp.mpf("1e-25")
            rest.pop(j)


def test_fp64_eigenvalues_are_meaningless_at_the_fig2_state():
    """(2, 30, 0, 1), dx = 3e-3, dt = tau = 1e-5 (Fig. 2): FP64 eigenvalues of the FP64 matrix are off
    by more than 1e-3, while 40 and 60 digits agree to 1e-15. max|omega| there is 1 + 7.18e-7."""
    st, xi, args = (2.0, 30.0, 0.0, 1.0), 0.3, (3e-3, 3e-3, 1e-5, 1e-5, 0.5)
    w40 = V.max_abs_eig_mp(st, xi, 0.0, *args, dps=40)
    w60 = V.max_abs_eig_mp(st, xi, 0.0, *args, dps=60)
    assert abs(w40 - w60) <= 1e-15
    assert abs(w40 - 1.0000007179897) <= 1e-12
    w64 = float(np.abs(np.linalg.eigvals(V.amplification_matrix(st, xi, 0.0, *args))).max())
    assert abs(w64 - w40) > 1e-3
