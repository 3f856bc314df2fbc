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

High precision (``*_mp``). At the high-Mach states of Sec. 4 the eigenvalues of
G are extremely sensitive: at (rho, u1, u2, T) = (2, 30, 0, 1) a relative
perturbation of G of 1e-16 moves them by O(1), while 1e-32 moves them by
1e-16. The entries of G carry the cancellation of the 4th-order f^eq at
s = v.u/theta ~ 135. So FP64 eigenvalues there mean nothing. The ``*_mp``
functions build G from Eqs. 10-13 and 18-20 in mpmath at ``dps`` decimal digits:
- f^eq is restated from Eq. 10;
- its T and u derivatives are taken by mpmath's numerical differentiation at
  that precision;
- the eigenvalues come from mpmath's QR.
The speeds are the binary64 values nearest 1, 1.92, 2.99, 4.49, converted
exactly, so the model is the one the C oracle and the CUDA library use. The
direction cosines are exact. The results hold to about dps - 20 digits at the
worst states of Sec. 4.
"""
import mpmath as mp
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


# ---------------------------------------------------------------------------------------------
# high precision (mpmath)

def _mp_velocities():
    """Eq. 1 with exact direction cosines: q = 1 + 8(k-1) + (i-1), direction i at angle i pi/4."""
    speeds = [mp.mpf(1.0), mp.mpf(1.92), mp.mpf(2.99), mp.mpf(4.49)]  # binary64 values, exactly
    vx, vy = [mp.mpf(0)], [mp.mpf(0)]
    for k in range(4):
        for i in range(1, 9):
            vx.append(speeds[k] * mp.cos(i * mp.pi / 4))
            vy.append(speeds[k] * mp.sin(i * mp.pi / 4))
    # cos/sin of multiples of pi/4 are 0, +-1 or +-sqrt(1/2): snap the zeros and ones exactly
    for v in (vx, vy):
        for q in range(1, Q):
            sp = speeds[(q - 1) // 8]
            r = v[q] / sp
            if abs(r) < mp.mpf(10) ** (-mp.mp.dps + 5):
                v[q] = mp.mpf(0)
            elif abs(abs(r) - 1) < mp.mpf(10) ** (-mp.mp.dps + 5):
                v[q] = sp * mp.sign(r)
    return speeds, vx, vy


def _mp_weights(speeds, theta):
    """(F_0, F_1..F_4) of Eqs. 11-13 with the cyclic index {k+l}."""
    F = []
    for k in range(4):
        vk2 = speeds[k] ** 2
        a, b, c = (speeds[(k + l) % 4] ** 2 for l in (1, 2, 3))
        denom = vk2 * (vk2 - a) * (vk2 - b) * (vk2 - c)
        F.append((48 * theta ** 4 - 6 * (a + b + c) * theta ** 3 + (a * b + b * c + c * a) * theta ** 2
                  - a * b * c / 4 * theta) / denom)
    return [1 - 8 * sum(F)] + F


def feq_mp(n, ux, uy, T, dps=50):
    """f^eq (33 mpf) of Eq. 10, all five terms inside n F_k [...], theta = T (m = 1)."""
    with mp.workdps(dps):
        speeds, vx, vy = _mp_velocities()
        return _feq_mp(speeds, vx, vy, mp.mpf(n), mp.mpf(ux), mp.mpf(uy), mp.mpf(T))


def _feq_mp(speeds, vx, vy, n, ux, uy, T):
    F = _mp_weights(speeds, T)
    u2 = ux * ux + uy * uy
    out = []
    for q in range(Q):
        Fk = F[0] if q == 0 else F[1 + (q - 1) // 8]
        vu = vx[q] * ux + vy[q] * uy
        br = (1 - u2 / (2 * T) + u2 * u2 / (8 * T * T)
              + (vu / T) * (1 - u2 / (2 * T))
              + vu * vu / (2 * T * T) * (1 - u2 / (2 * T))
              + vu ** 3 / (6 * T ** 3) + vu ** 4 / (24 * T ** 4))
        out.append(n * Fk * br)
    return out


def amplification_matrix_mp(state, kx_dx, ky_dy, dx, dy, dt, tau, lam=0.0,
                            lw=True, disp=True, visc=True, dps=50):
    """G of Eq. 18 (mpmath matrix at dps digits); same terms and switches as amplification_matrix."""
    with mp.workdps(dps):
        speeds, vx, vy = _mp_velocities()
        n, ux, uy, T = (mp.mpf(x) for x in state)
        fe = _feq_mp(speeds, vx, vy, n, ux, uy, T)
        dT = [mp.diff(lambda t, q=q: _feq_mp(speeds, vx, vy, n, ux, uy, t)[q], T) for q in range(Q)]
        dux = [mp.diff(lambda a, q=q: _feq_mp(speeds, vx, vy, n, a, uy, T)[q], ux) for q in range(Q)]
        duy = [mp.diff(lambda a, q=q: _feq_mp(speeds, vx, vy, n, ux, a, T)[q], uy) for q in range(Q)]
        r = mp.mpf(dt) / mp.mpf(tau)
        G = mp.matrix(Q, Q)
        for j in range(Q):
            wx, wy = vx[j] - ux, vy[j] - uy
            cT = ((wx * wx + wy * wy) / 2 - T) / n
            for i in range(Q):  # Eq. 20
                G[i, j] = r * (fe[i] / n + dT[i] * cT + dux[i] * wx / n + duy[i] * wy / n)
        for i in range(Q):
            G[i, i] += 1 - r
            for xi, va, dr, ua in ((mp.mpf(kx_dx), vx, mp.mpf(dx), ux), (mp.mpf(ky_dy), vy, mp.mpf(dy), uy)):
                c = va[i] * mp.mpf(dt) / dr
                e1, e2 = mp.expj(xi), mp.expj(2 * xi)
                d = -(c / 2) * (e1 - 1 / e1)
                if lw:
                    d += (c * c / 2) * (e1 - 2 + 1 / e1)
                if disp:
                    d += c * (1 - c * c) / 12 * (e2 - 2 * e1 + 2 / e1 - 1 / e2)
                if visc:
                    kap = abs(ua * mp.mpf(dt) / dr)
                    d += mp.mpf(lam) * kap * (1 - kap) / 2 * (e1 - 2 + 1 / e1)
                G[i, i] += d
        return G


def eigvals_mp(G, dps=50):
    """The 33 eigenvalues of an mpmath matrix, as mpc, by mpmath's QR at dps digits."""
    with mp.workdps(dps):
        return list(mp.eig(G, left=False, right=False))


def max_abs_eig_mp(state, kx_dx, ky_dy, dx, dy, dt, tau, lam=0.0, dps=50, **kw):
    """max |omega| of G (Eq. 18) at dps digits, returned as a float."""
    G = amplification_matrix_mp(state, kx_dx, ky_dy, dx, dy, dt, tau, lam, dps=dps, **kw)
    with mp.workdps(dps):
        return float(max(abs(z) for z in eigvals_mp(G, dps)))
