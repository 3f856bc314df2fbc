"""Pins of the oracle's velocity set, weights and equilibrium (Sec. 2, Eqs. 1, 3-5, 10-13).

Each check compares the oracle with something other than its own formulas:
trigonometric closed forms for the 8-direction rings, the radial moments of
the 2-D Maxwellian (a generic linear solve), and Maxwellian moments computed
by Gauss-Hermite quadrature.
"""
import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial.hermite_e import hermegauss

from oracle import fdlbm as O

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_states.json")))


def test_velocity_set_geometry():
    """Eq. 1: q = 1 + 8(k-1) + (i-1) has speed v_k and angle i*pi/4; rest velocity at q = 0."""
    vx, vy = O.velocities()
    speeds = GOLDEN["speeds"]["v"]
    assert vx[0] == 0.0 and vy[0] == 0.0
    for k in range(1, 5):
        for i in range(1, 9):
            q = 1 + 8 * (k - 1) + (i - 1)
            assert math.hypot(vx[q], vy[q]) == pytest.approx(speeds[k], rel=1e-15)
            ang = math.atan2(vy[q], vx[q]) % (2 * math.pi)
            assert ang == pytest.approx((i * math.pi / 4) % (2 * math.pi), abs=1e-15)
    # axis directions carry exact zeros (cos(pi/2) is not evaluated)
    for k in range(1, 5):
        assert vy[1 + 8 * (k - 1) + 7] == 0.0 and vx[1 + 8 * (k - 1) + 1] == 0.0


def test_ring_isotropy_closed_forms():
    """Sums over the 8 directions of one ring: the closed forms of sum_i cos^a sin^b (i pi/4)."""
    vx, vy = O.velocities()
    ex, ey = vx[1:9] / 1.0, vy[1:9] / 1.0  # ring k = 1 has unit speed
    th = np.arange(1, 9) * np.pi / 4
    closed = {  # exact trigonometric sums over 8 equally spaced angles
        (2, 0): 4.0, (0, 2): 4.0, (1, 1): 0.0, (4, 0): 3.0, (2, 2): 1.0, (0, 4): 3.0,
        (6, 0): 2.5, (4, 2): 0.5, (2, 4): 0.5, (1, 0): 0.0, (3, 0): 0.0, (2, 1): 0.0, (5, 0): 0.0,
        (3, 3): 0.0, (5, 1): 0.0, (7, 0): 0.0,
    }
    for (a, b), val in closed.items():
        assert np.sum(ex ** a * ey ** b) == pytest.approx(val, abs=1e-14)
        assert np.sum(np.cos(th) ** a * np.sin(th) ** b) == pytest.approx(val, abs=1e-14)


@pytest.mark.parametrize("theta", [0.05, 0.5, 1.0, 7.928, 22.61, 178.555, 1000.0])
def test_weights_match_maxwellian_radial_moments(theta):
    """Eqs. 11-12 against a generic solve of sum_k 8 F_k v_k^(2m) = E|v|^(2m) = 2^m m! theta^m.

    E|v|^(2m) of a unit-density 2-D Maxwellian with temperature theta is (2 theta)^m m!.
    Eq. 12 then fixes F_0 so the weights sum to one."""
    F = O.weights(theta)
    v = np.array(GOLDEN["speeds"]["v"][1:])
    A = np.array([[8.0 * v[k] ** (2 * m) for k in range(4)] for m in range(1, 5)])
    b = np.array([(2.0 * theta) ** m * math.factorial(m) for m in range(1, 5)])
    Fs = np.linalg.solve(A, b)
    scale = np.abs(Fs).max()
    assert np.max(np.abs(F[1:] - Fs)) <= 1e-12 * scale
    assert F[0] + 8.0 * F[1:].sum() == pytest.approx(1.0, abs=1e-13 * max(1.0, 8 * scale))


def _maxwell_moment(n, ux, uy, T, a, b, c):
    """n E[vx^a vy^b |v|^(2c)] for v ~ N(u, T I): 40-point Gauss-Hermite in each axis."""
    x, w = hermegauss(40)
    w = w / math.sqrt(2.0 * math.pi)
    X = ux + math.sqrt(T) * x[:, None]
    Y = uy + math.sqrt(T) * x[None, :]
    return n * np.sum((w[:, None] * w[None, :]) * X ** a * Y ** b * (X * X + Y * Y) ** c)


EXACT_MOMENTS = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 0, 0), (1, 1, 0), (0, 2, 0), (3, 0, 0), (2, 1, 0),
                 (1, 2, 0), (0, 3, 0), (2, 0, 1), (1, 1, 1), (0, 2, 1), (0, 0, 2), (1, 0, 1), (0, 1, 1)]

STATES = [(1.0, 0.0, 0.0, 1.0), (1.3, 0.4, -0.2, 0.7), (0.125, 0.0, 0.0, 0.8),
          (0.445, 0.698, 0.0, 7.928), (1.0, 20.0, 0.0, 0.5), (50.0 / 17.0, 16.7, -5.71578, 22.61),
          (5.99924, 19.5975, 0.0, 76.8254), (2.0, 0.0, -3.0, 0.05)]


@pytest.mark.parametrize("state", STATES)
def test_feq_reproduces_maxwellian_moments(state):
    """Eq. 10 (all five bracket terms inside nF_k[...]): the moments through third order, the
    contracted fourth-order moments |v|^2 v_a v_b and |v|^4, equal those of the Maxwellian.
    Error bound: a few ulps of sum_q |f_eq phi| (the conditioning kappa of the state)."""
    fe = O.feq(*state)
    vx, vy = O.velocities()
    for (a, b, c) in EXACT_MOMENTS:
        phi = vx ** a * vy ** b * (vx * vx + vy * vy) ** c
        disc = np.sum(fe * phi)
        cont = _maxwell_moment(*state, a, b, c)
        scale = np.sum(np.abs(fe * phi)) + abs(cont)
        assert abs(disc - cont) <= 64 * np.finfo(float).eps * scale, (a, b, c, disc, cont)


def test_feq_is_not_a_full_fourth_order_maxwellian():
    """Control: vx^4 (uncontracted 4th order) is not reproduced at u != 0, so the moment
    test above can tell the exact moments from the rest."""
    state = (1.3, 0.4, -0.2, 0.7)
    fe = O.feq(*state)
    vx, vy = O.velocities()
    disc = np.sum(fe * vx ** 4)
    cont = _maxwell_moment(*state, 4, 0, 0)
    assert abs(disc - cont) > 1e-6 * abs(cont)


@pytest.mark.parametrize("state", STATES)
def test_moments_invert_feq(state):
    """Eqs. 3-5 applied to f_eq(n, u, T) return (n, u, T)."""
    fe = O.feq(*state)
    n, ux, uy, T = O.moments(fe)
    kappa = np.abs(fe).sum() / state[0]
    tol = 1e-13 * kappa
    u_scale = max(1.0, abs(state[1]), abs(state[2]))
    assert n == pytest.approx(state[0], rel=tol)
    assert abs(ux - state[1]) <= tol * u_scale and abs(uy - state[2]) <= tol * u_scale
    assert T == pytest.approx(state[3], rel=tol * max(1.0, (state[1] ** 2 + state[2] ** 2) / state[3]))


def test_feq_rest_state_is_weights():
    """At u = 0 the bracket of Eq. 10 is 1, so f_eq = n F_k."""
    fe = O.feq(2.0, 0.0, 0.0, 1.7)
    F = O.weights(1.7)
    assert fe[0] == pytest.approx(2.0 * F[0], rel=1e-15)
    for q in range(1, 33):
        assert fe[q] == pytest.approx(2.0 * F[1 + (q - 1) // 8], rel=1e-15)
