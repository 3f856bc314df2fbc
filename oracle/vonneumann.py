"""von Neumann amplification matrix of Sec. 4 (Eqs. 18-20); test infrastructure only.

G(k) is the 33 x 33 matrix that maps the Fourier amplitude of a small
perturbation of a uniform equilibrium state from one time step to the next:

  G_ij = (1 - dt/tau) delta_ij + (dt/tau) d f_i^eq / d f_j
         + delta_ij sum_alpha [ -(c_ia/2)(e^{i xi} - e^{-i xi})
                                + (c_ia^2/2)(e^{i xi} - 2 + e^{-i xi})
                                + c_ia (1 - c_ia^2)/12 (e^{2i xi} - 2 e^{i xi} + 2 e^{-i xi} - e^{-2i xi})
                                + theta_a |kappa_a| (1 - |kappa_a|)/2 (e^{i xi} - 2 + e^{-i xi}) ]

with xi = k_alpha * dr_alpha (Eq. 18), and the equilibrium Jacobian taken
through rho, T and u_alpha (Eq. 20):

  d f_i^eq / d f_j = f_i^eq/rho + (d f_i^eq/dT)(|v_j - u|^2/2 - T)/rho
                     + sum_alpha (d f_i^eq/d u_alpha)(v_ja - u_alpha)/rho .

The partial derivatives of f^eq in T and u are taken numerically from the
oracle's f^eq (Eq. 10) by Richardson-extrapolated central differences.

Reading: the switch theta_alphaI of Eq. 16 is quadratic in a perturbation
and drops out of a linearisation, yet Sec. 4 varies lambda, so the analysis
holds theta_alphaI at lambda (the oracle's SWITCH_CONST flag is the matching
simulation).
"""
import numpy as np

from . import fdlbm as _o

Q = 33


def _d(fun, x, h):
    """Richardson-extrapolated central difference of a vector function."""
    d1 = (fun(x + h) - fun(x - h)) / (2.0 * h)
    d2 = (fun(x + h / 2.0) - fun(x - h / 2.0)) / h
    return (4.0 * d2 - d1) / 3.0


def feq_jacobian(rho, ux, uy, T):
    """d f^eq_i / d f_j (33 x 33) of Eq. 20."""
    vx, vy = _o.velocities()
    fe = _o.feq(rho, ux, uy, T)
    dT = _d(lambda t: _o.feq(rho, ux, uy, t), T, 1e-4 * T)
    hu = 1e-4 * max(1.0, abs(ux), abs(uy))
    dux = _d(lambda a: _o.feq(rho, a, uy, T), ux, hu)
    duy = _d(lambda a: _o.feq(rho, ux, a, T), uy, hu)
    wx = vx - ux
    wy = vy - uy
    dT_df = (0.5 * (wx * wx + wy * wy) - T) / rho
    dux_df = wx / rho
    duy_df = wy / rho
    J = (fe / rho)[:, None] * np.ones(Q)[None, :]
    J += dT[:, None] * dT_df[None, :]
    J += dux[:, None] * dux_df[None, :]
    J += duy[:, None] * duy_df[None, :]
    return J


def amplification_matrix(state, kx_dx, ky_dy, dx, dy, dt, tau, lam=0.0,
                         lw=True, disp=True, visc=True, J=None):
    """G of Eq. 18 for uniform state (rho, u1, u2, T) at wave numbers xi_x = kx*dx, xi_y = ky*dy.

    lw/disp/visc switch lines II/III/IV of Eq. 17 (the Sec. 4 scheme variants);
    the switch theta_alphaI is held at lam.
    """
    rho, ux, uy, T = state
    vx, vy = _o.velocities()
    if J is None:
        J = feq_jacobian(rho, ux, uy, T)
    r = dt / tau
    G = (1.0 - r) * np.eye(Q, dtype=complex) + r * J.astype(complex)
    diag = np.zeros(Q, dtype=complex)
    for xi, va, dr, ua in ((kx_dx, vx, dx, ux), (ky_dy, vy, dy, uy)):
        c = va * dt / dr
        e1, e2 = np.exp(1j * xi), np.exp(2j * xi)
        diag += -(c / 2.0) * (e1 - 1.0 / e1)
        if lw:
            diag += (c * c / 2.0) * (e1 - 2.0 + 1.0 / e1)
        if disp:
            diag += c * (1.0 - c * c) / 12.0 * (e2 - 2.0 * e1 + 2.0 / e1 - 1.0 / e2)
        if visc:
            kap = ua * dt / dr
            diag += lam * abs(kap) * (1.0 - abs(kap)) / 2.0 * (e1 - 2.0 + 1.0 / e1)
    G += np.diag(diag)
    return G


def max_abs_eig(G):
    return float(np.max(np.abs(np.linalg.eigvals(G))))


def max_growth(state, dx, dy, dt, tau, lam=0.0, nk=64, axis="x", **kw):
    """max over k dx in (0, pi] of max|omega| (the curves of Figs. 2, 4-6)."""
    J = feq_jacobian(*state)
    best = 0.0
    for xi in np.linspace(np.pi / nk, np.pi, nk):
        kx, ky = (xi, 0.0) if axis == "x" else (0.0, xi)
        best = max(best, max_abs_eig(amplification_matrix(state, kx, ky, dx, dy, dt, tau, lam, J=J, **kw)))
    return best
