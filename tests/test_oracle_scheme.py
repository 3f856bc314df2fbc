"""Pins of the oracle's time step (Sec. 3, Eqs. 15-17) and boundary fill.

The checks rest on facts the paper and the mathematics fix, not on the
oracle's own formulas: fixed points, exact decay laws, symmetries, discrete
conservation, the convergence order of the advection stencil, the paper's
amplification matrix (Eq. 18), and a mirror construction for the wall.
"""
import math

import numpy as np
import pytest

from oracle import fdlbm as O
from oracle import vonneumann as V

PER = (O.PERIODIC,) * 4


def _smooth_fields(nx, ny, seed, amp=0.1, base=(1.0, 0.3, -0.2, 1.0)):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * (np.arange(nx) + 0.5) / nx
    y = 2 * np.pi * (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for b in base:
        a1, a2, p1, p2 = rng.uniform(-1, 1, 4)
        out.append(b + amp * (abs(b) + 0.5) * (a1 * np.sin(X + p1) + a2 * np.cos(Y + 2 * X + p2)))
    return out


@pytest.mark.parametrize("state", [(1.0, 0.0, 0.0, 1.0), (1.3, 0.4, -0.2, 0.7), (1.0, 20.0, 0.0, 0.5),
                                   (50.0 / 17.0, 16.7, -5.71578, 22.61)])
def test_uniform_state_is_fixed_point(state):
    """A uniform equilibrium has zero differences (lines I-IV vanish) and f = f_eq(moments(f))."""
    nx, ny = 6, 5
    s = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 2e-5, 1.0, PER)
    s.set_macro(*[np.full((ny, nx), c) for c in state])
    f0 = s.get_f()
    assert s.step(50) == 0
    f1 = s.get_f()
    kappa = np.abs(O.feq(*state)).sum() / state[0]
    assert np.max(np.abs(f1 - f0)) <= 1e-14 * kappa * np.max(np.abs(f0)) * 50
    # the differences are exactly zero, so every node stays bitwise equal to every other
    assert np.all(f1 == f1[:, :1, :1])


def test_relaxation_decay_law():
    """Uniform non-equilibrium f: stencil terms vanish and relaxation conserves n, nu, E, so
    f - f_eq decays exactly as (1 - dt/tau)^n (Eq. 17 line I, relaxation counted once)."""
    nx, ny = 4, 3
    dt, tau = 1e-5, 4e-5
    vx, vy = O.velocities()
    state = (1.2, 0.3, 0.1, 0.9)
    fe = O.feq(*state)
    rng = np.random.default_rng(0)
    d = rng.normal(size=33)
    # remove the components along the collision invariants 1, vx, vy, |v|^2
    B = np.stack([np.ones(33), vx, vy, vx * vx + vy * vy], 1)
    d -= B @ np.linalg.lstsq(B, d, rcond=None)[0]
    d *= 1e-3
    s = O.Sim(nx, ny, 1e-3, 1e-3, dt, tau, 2.0, PER)
    s.set_f(np.broadcast_to((fe + d)[:, None, None], (33, ny, nx)))
    nsteps = 7
    assert s.step(nsteps) == 0
    f = s.get_f()[:, 0, 0]
    expect = fe + (1.0 - dt / tau) ** nsteps * d
    assert np.max(np.abs(f - expect)) <= 1e-13 * np.abs(fe).max()


def test_y_uniform_fields_stay_y_uniform_bitwise():
    """y-differences of identical rows are exactly zero: a 2-D run on y-uniform data equals
    the ny = 1 run row by row, bit for bit."""
    nx = 40
    rho, u, v, T = [a[0] for a in _smooth_fields(nx, 1, 3)]
    s1 = O.Sim(nx, 1, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, (O.OUTFLOW, O.OUTFLOW, O.PERIODIC, O.PERIODIC))
    s4 = O.Sim(nx, 4, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, (O.OUTFLOW, O.OUTFLOW, O.PERIODIC, O.PERIODIC))
    s1.set_macro(rho[None], u[None], v[None], T[None])
    s4.set_macro(*[np.repeat(a[None], 4, 0) for a in (rho, u, v, T)])
    assert s1.step(30) == 0 and s4.step(30) == 0
    f1, f4 = s1.get_f(), s4.get_f()
    for j in range(4):
        assert np.array_equal(f4[:, j, :], f1[:, 0, :])


def _transpose_q():
    """velocity index under the reflection (x, y) -> (y, x): direction i -> 2 - i (mod 8)."""
    perm = [0]
    for k in range(1, 5):
        for i in range(1, 9):
            j = (2 - i) % 8
            j = 8 if j == 0 else j
            perm.append(1 + 8 * (k - 1) + (j - 1))
    return np.array(perm)


def test_transpose_symmetry():
    """Swapping x <-> y (with u <-> v) commutes with the step on a square periodic grid."""
    n = 12
    rho, u, v, T = _smooth_fields(n, n, 5, amp=0.15)
    a = O.Sim(n, n, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, PER)
    b = O.Sim(n, n, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, PER)
    a.set_macro(rho, u, v, T)
    b.set_macro(rho.T.copy(), v.T.copy(), u.T.copy(), T.T.copy())
    assert a.step(20) == 0 and b.step(20) == 0
    fa, fb = a.get_f(), b.get_f()
    perm = _transpose_q()
    fa_t = np.transpose(fa, (0, 2, 1))[perm]
    assert np.max(np.abs(fa_t - fb)) <= 1e-13 * np.abs(fa).max()


@pytest.mark.parametrize("base", [(1.0, 0.3, -0.2, 1.0), (1.0, 2.0, 1.0, 0.8)])
def test_conservation_at_lambda_zero(base):
    """With lambda = 0 every term of Eq. 17 is a constant-coefficient difference or a collision
    term with zero mass, momentum and energy moments: the totals are conserved on a periodic
    grid to rounding."""
    nx, ny = 16, 12
    s = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 0.0, PER)
    s.set_macro(*_smooth_fields(nx, ny, 7, amp=0.1, base=base))
    vx, vy = O.velocities()

    def totals():
        f = s.get_f().sum(axis=(1, 2))
        return np.array([f.sum(), (vx * f).sum(), (vy * f).sum(), (0.5 * (vx * vx + vy * vy) * f).sum()])

    t0 = totals()
    assert s.step(40) == 0
    t1 = totals()
    fe_scale = np.abs(s.get_f()).sum()
    assert np.max(np.abs(t1 - t0)) <= 1e-13 * fe_scale * 40


def test_viscosity_breaks_conservation_only_through_line_iv():
    """Control for the test above: with lambda > 0 line IV has a node-varying coefficient and
    mass changes; without line IV (NO_VISC) it is conserved again."""
    nx, ny = 16, 12
    fields = _smooth_fields(nx, ny, 9, amp=0.3)
    masses = []
    for lam, flags in [(2.0, 0), (2.0, O.NO_VISC)]:
        s = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, lam, PER, flags=flags)
        s.set_macro(*fields)
        m0 = s.get_f().sum()
        assert s.step(40) == 0
        masses.append(abs(s.get_f().sum() - m0) / m0)
    assert masses[0] > 1e-9 and masses[1] < 1e-13


def _advection_error(nx, q, cfl_cells):
    """Advect a smooth wave carried by velocity q alone (collision negligible, lambda = 0) over a
    fixed physical time on a periodic line; return the max error against exact translation."""
    vx, vy = O.velocities()
    L = 1.0
    dx = L / nx
    dt = cfl_cells * dx / 4.49
    nsteps = int(round(0.25 / dt))
    dt = 0.25 / nsteps
    base = O.feq(1.0, 0.0, 0.0, 1.0)
    x = (np.arange(nx) + 0.5) * dx
    amp = 1e-3
    f = np.broadcast_to(base[:, None, None], (33, 1, nx)).copy()
    f[q, 0, :] += amp * np.sin(2 * np.pi * x / L)
    s = O.Sim(nx, 1, dx, dx, dt, 1e30, 0.0, PER)
    s.set_f(f)
    assert s.step(nsteps) == 0
    got = s.get_f()[q, 0, :] - base[q]
    exact = amp * np.sin(2 * np.pi * (x - vx[q] * nsteps * dt) / L)
    return np.max(np.abs(got - exact)) / amp


@pytest.mark.parametrize("q", [32, 28, 25])
def test_advection_is_third_order(q):
    """Lines I-III of Eq. 17 form a third-order scheme for v df/dx: the dispersion line cancels
    the Lax-Wendroff phase error, so halving dx (fixed Courant number) cuts the error ~8x.
    q = 32 is +x at the top speed, 28 is -x, 25 the 45-degree direction."""
    e1 = _advection_error(64, q, 0.5)
    e2 = _advection_error(128, q, 0.5)
    order = math.log2(e1 / e2)
    assert 2.7 < order < 3.3, order


def _linearised_step(state, nx, ny, mode, dx, dy, dt, tau, lam, flags):
    """Build the one-step linear map of the oracle on Fourier mode (mx, my) column by column."""
    fe = O.feq(*state)
    eps = 1e-6 * np.abs(fe).max()
    ii = np.arange(nx)[None, :]
    jj = np.arange(ny)[:, None]
    ph = 2 * np.pi * (mode[0] * ii / nx + mode[1] * jj / ny)
    G = np.zeros((33, 33), complex)
    for j in range(33):
        outs = []
        for sgn in (1.0, -1.0):
            s = O.Sim(nx, ny, dx, dy, dt, tau, lam, PER, flags=flags)
            f = np.broadcast_to(fe[:, None, None], (33, ny, nx)).copy()
            f[j] += sgn * eps * np.cos(ph)
            s.set_f(f)
            assert s.step(1) == 0
            outs.append(s.get_f())
        d = (outs[0] - outs[1]) / (2 * eps)
        c = np.sum(d * np.cos(ph)[None], axis=(1, 2)) * 2.0 / (nx * ny)
        sn = np.sum(d * np.sin(ph)[None], axis=(1, 2)) * 2.0 / (nx * ny)
        G[:, j] = c - 1j * sn
    return G


@pytest.mark.parametrize("mode,shape", [((1, 0), (8, 1)), ((3, 0), (8, 1)), ((0, 1), (1, 8)), ((1, 1), (8, 8))])
@pytest.mark.parametrize("lam,flags", [(0.5, O.SWITCH_CONST), (0.0, 0)])
def test_linearised_step_equals_amplification_matrix(mode, shape, lam, flags):
    """The oracle's step, linearised about a uniform equilibrium, equals G of Eq. 18 with the
    Jacobian of Eq. 20, element by element (switch held at lambda, Sec. 4 reading)."""
    state = (1.0, 0.3, -0.2, 1.0)
    dx, dy, dt, tau = 3e-3, 2e-3, 1e-5, 2e-5
    nx, ny = shape
    Gs = _linearised_step(state, nx, ny, mode, dx, dy, dt, tau, lam, flags)
    xi_x = 2 * np.pi * mode[0] / nx
    xi_y = 2 * np.pi * mode[1] / ny
    Gp = V.amplification_matrix(state, xi_x, xi_y, dx, dy, dt, tau, lam)
    assert np.max(np.abs(Gs - Gp)) <= 1e-7 * np.abs(Gp).max()


def test_switch_vanishes_in_linearisation():
    """theta_alphaI of Eq. 16 is O(perturbation): with the pressure switch on, the linear map
    is that of lambda = 0 (up to O(eps))."""
    state = (1.0, 0.3, -0.2, 1.0)
    Gs = _linearised_step(state, 8, 1, (1, 0), 3e-3, 3e-3, 1e-5, 1e-5, 5.0, 0)
    Gp = V.amplification_matrix(state, 2 * np.pi / 8, 0.0, 3e-3, 3e-3, 1e-5, 1e-5, 0.0)
    assert np.max(np.abs(Gs - Gp)) <= 1e-5 * np.abs(Gp).max()


def test_stability_claims_of_sec4():
    """Sec. 4 claims (Fig. 2): Lax-Wendroff favours stability, dispersion disfavours it, and the
    artificial viscosity brings max|omega| to <= 1. Checked at (1, 10, 0, 1), dx = 3e-3,
    dt = tau = 1e-5, lambda = 0.5 (the Fig. 2 state itself is too ill-conditioned, kappa ~ 1e5)."""
    st = (1.0, 10.0, 0.0, 1.0)
    args = (3e-3, 3e-3, 1e-5, 1e-5)
    central = V.max_growth(st, *args, lam=0.5, nk=48, lw=False, disp=False, visc=False)
    lw = V.max_growth(st, *args, lam=0.5, nk=48, lw=True, disp=False, visc=False)
    disp = V.max_growth(st, *args, lam=0.5, nk=48, lw=False, disp=True, visc=False)
    full = V.max_growth(st, *args, lam=0.5, nk=48)
    assert lw < central < disp
    assert central > 1.0 and full <= 1.0 + 1e-12


def test_growth_increases_with_velocity():
    """Sec. 4 (Fig. 6): at lambda = 0 the largest eigenvalue grows with u1. FP64 eigenvalues are
    trustworthy to ~1e-5 only up to u1 ~ 15 at T = 1 (see the high-precision tests), so the max
    over k is taken in FP64 there, and the higher velocities are compared at one wave number in
    50-digit arithmetic."""
    vals = [V.max_growth((2.0, u, 0.0, 1.0), 3e-3, 3e-3, 1e-5, 1e-5, lam=0.0, nk=48) for u in (5, 10, 15)]
    assert all(b > a for a, b in zip(vals, vals[1:]))
    hp = [V.max_abs_eig_mp((2.0, u, 0.0, 1.0), 1.5, 0.0, 3e-3, 3e-3, 1e-5, 1e-5, 0.0, dps=40) for u in (15, 20, 30)]
    assert all(b > a for a, b in zip(hp, hp[1:]))


def test_wall_equals_mirrored_periodic_domain():
    """Specular walls at bottom and top: the solution equals the lower half of a periodic domain
    of twice the height whose upper half is the mirror image (v -> -v). Mirrored nodes sum
    their moments over a permuted q order, so the two agree to rounding, not bitwise."""
    nx, ny = 10, 6
    rho, u, v, T = _smooth_fields(nx, ny, 11, amp=0.1, base=(1.0, 0.4, 0.0, 1.0))
    v = 0.2 * np.sin(np.pi * (np.arange(ny)[:, None] + 0.5) / ny) * np.ones((ny, nx))
    w = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, (O.PERIODIC, O.PERIODIC, O.WALL, O.WALL))
    w.set_macro(rho, u, v, T)
    p = O.Sim(nx, 2 * ny, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, PER)
    p.set_macro(np.vstack([rho, rho[::-1]]), np.vstack([u, u[::-1]]), np.vstack([v, -v[::-1]]),
                np.vstack([T, T[::-1]]))
    assert w.step(25) == 0 and p.step(25) == 0
    fw, fp = w.get_f(), p.get_f()
    assert np.max(np.abs(fw - fp[:, :ny, :])) <= 1e-13 * np.abs(fw).max()
    # control: a wall that does not reverse v is far from the mirror solution
    assert np.max(np.abs(fw - fp[:, ny:, :][:, ::-1, :])) > 1e-6 * np.abs(fw).max()


def test_x_wall_equals_mirrored_periodic_domain():
    """Same construction along x (left/right walls, u -> -u), to rounding."""
    nx, ny = 6, 5
    rho, u, v, T = _smooth_fields(nx, ny, 12, amp=0.1, base=(1.0, 0.0, 0.3, 1.0))
    w = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, (O.WALL, O.WALL, O.PERIODIC, O.PERIODIC))
    w.set_macro(rho, u, v, T)
    p = O.Sim(2 * nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, PER)
    p.set_macro(np.hstack([rho, rho[:, ::-1]]), np.hstack([u, -u[:, ::-1]]), np.hstack([v, v[:, ::-1]]),
                np.hstack([T, T[:, ::-1]]))
    assert w.step(25) == 0 and p.step(25) == 0
    fw, fp = w.get_f(), p.get_f()
    assert np.max(np.abs(fw - fp[:, :, :nx])) <= 1e-13 * np.abs(fw).max()


def test_ghost_ring_contents():
    """Outflow ghosts copy the edge node; Dirichlet ghosts hold f_eq of the side's state;
    periodic ghosts wrap."""
    nx, ny = 7, 5
    bstate = np.zeros((4, 4))
    bstate[3] = (1.5, 0.2, -0.1, 0.9)
    s = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 1.0, (O.PERIODIC, O.PERIODIC, O.OUTFLOW, O.DIRICHLET), bstate)
    s.set_macro(*_smooth_fields(nx, ny, 13))
    s.step(3)
    g = s.get_f_padded()  # [q][j+2][i+2]
    I = slice(2, 2 + nx)
    assert np.array_equal(g[:, 0, I], g[:, 2, I]) and np.array_equal(g[:, 1, I], g[:, 2, I])
    fe = O.feq(*bstate[3])
    assert np.array_equal(g[:, ny + 2, I], np.broadcast_to(fe[:, None], (33, nx)))
    assert np.array_equal(g[:, ny + 3, I], np.broadcast_to(fe[:, None], (33, nx)))
    J = slice(2, 2 + ny)
    assert np.array_equal(g[:, J, 0], g[:, J, nx]) and np.array_equal(g[:, J, 1], g[:, J, nx + 1])
    assert np.array_equal(g[:, J, nx + 2], g[:, J, 2]) and np.array_equal(g[:, J, nx + 3], g[:, J, 3])


def test_bad_state_is_reported():
    """A negative temperature makes P <= 0, where Eq. 16 is undefined: the step reports -4."""
    s = O.Sim(5, 3, 1e-3, 1e-3, 1e-5, 1e-5, 1.0, PER)
    T = np.ones((3, 5))
    s.set_macro(np.ones((3, 5)), np.zeros((3, 5)), np.zeros((3, 5)), T)
    f = s.get_f()
    f[0, 1, 2] -= 5.0  # drives n T negative at one node
    s.set_f(f)
    assert s.step(1) == -4


def _switch_theta(rho, u, T, lam=1.0, dx=1e-3, dt=1e-5):
    """theta_xI of Eq. 16 read back from one oracle step on a line (ny = 1).

    f(lam, switch) - f(0) = theta_I * L and f(1, switch held at 1) - f(0) = L, where L is the rest
    of line IV (pinned by the amplification-matrix test), so their ratio is theta_I / 1."""
    nx = len(rho)
    outs = {}
    for key, lm, fl in (("off", 0.0, 0), ("sw", lam, 0), ("one", 1.0, O.SWITCH_CONST)):
        s = O.Sim(nx, 1, dx, dx, dt, dt, lm, (O.PERIODIC,) * 4, flags=fl)
        s.set_macro(rho[None], u[None], np.zeros((1, nx)), T[None])
        assert s.step(1) == 0
        outs[key] = s.get_f()[:, 0, :]
    d_sw = outs["sw"] - outs["off"]
    d_one = outs["one"] - outs["off"]
    q = np.argmax(np.abs(d_one), axis=0)
    cols = np.arange(nx)
    return d_sw[q, cols] / d_one[q, cols]


def test_switch_uses_pressure_and_is_bounded():
    """Eq. 16 structure: theta = 0 where P is uniform (even with rho and T varying) or affine in x,
    0 <= theta <= lambda for any positive P, and theta is unchanged when P is scaled."""
    nx = 12
    x = np.arange(nx)
    u = np.full(nx, 0.5)
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x / nx)
    th = _switch_theta(rho, u, 1.0 / rho)  # P = rho T = 1 everywhere
    assert np.max(np.abs(th)) < 1e-9
    P = np.array([0.1, 1.0, 0.1, 0.5, 2.0, 0.3, 0.3, 1.5, 0.05, 1.0, 0.7, 0.2])
    lam = 1.7
    th = _switch_theta(np.ones(nx), u, P, lam=lam)
    assert np.all(th >= -1e-9) and np.all(th <= lam * (1 + 1e-9))
    assert th[1] > 0.5 * lam  # the spike P = (0.1, 1, 0.1) switches strongly
    th2 = _switch_theta(np.full(nx, 3.0), u, P, lam=lam)  # P -> 3 P
    assert np.max(np.abs(th2 - th)) < 1e-8 * lam
    Paff = 1.0 + 0.05 * np.minimum(x, nx - 1 - x)  # affine except at the two kinks
    th = _switch_theta(np.ones(nx), u, Paff, lam=lam)
    kinks = {0, nx - 1, (nx - 1) // 2, nx // 2}
    for i in range(nx):
        if i not in kinks:
            assert abs(th[i]) < 1e-9
