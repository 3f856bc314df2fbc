"""Exact solution of the 1-D Riemann problem for an ideal gas (test infrastructure only).

The paper compares its shock tubes (Sec. 5.1: Sod, Lax, Sjogreen, Colella,
two-shock collision) with "exact solutions" whose solver it does not print.
This module writes one from the gas-dynamics equations: the star-region
pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the
Rankine-Hugoniot (shock) or isentropic (rarefaction) relation between state K
and the star state, followed by sampling of the self-similar solution at x/t.

The model's ratio of specific heats is gamma = 2: in two dimensions the
internal energy is e_int = nT = P (Eq. 5), i.e. D/2 = 1 degree of freedom per
direction and gamma = (D + 2)/D = 2. The paper's own post-shock data (Eqs. 26,
27) reproduce gamma = 2 Rankine-Hugoniot states, which the tests check.
States are (rho, u, p); p = rho T with m = 1.
"""
import math

import numpy as np

GAMMA = 2.0


def _fk(p, rho, pk, ck, g):
    """f_K(p) and its derivative (shock branch if p > p_K, rarefaction otherwise)."""
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        sq = math.sqrt(A / (p + B))
        f = (p - pk) * sq
        df = sq * (1.0 - 0.5 * (p - pk) / (B + p))
    else:
        pr = p / pk
        f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=GAMMA, tol=1e-14, maxit=200):
    """(p*, u*) between left=(rho,u,p) and right=(rho,u,p). Raises if vacuum forms."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("initial data generate a vacuum")
    # two-rarefaction guess, then Newton
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-14 * min(pl, pr))
    for _ in range(maxit):
        fl, dfl = _fk(p, rl, pl, cl, g)
        fr, dfr = _fk(p, rr, pr, cr, g)
        dp = (fl + fr + (ur - ul)) / (dfl + dfr)
        pn = p - dp
        if pn <= 0.0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def vacuum_forms(left, right, g=GAMMA):
    """True if the data separate into two rarefactions with vacuum between them:
    2 (c_L + c_R)/(gamma - 1) <= u_R - u_L."""
    cl = math.sqrt(g * left[2] / left[0])
    cr = math.sqrt(g * right[2] / right[0])
    return 2.0 * (cl + cr) / (g - 1.0) <= right[1] - left[1]


def _sample_vacuum(left, right, xi, g):
    """Two rarefactions fanning into vacuum: the left fan ends at u_L + 2 c_L/(gamma-1), the
    right one begins at u_R - 2 c_R/(gamma-1); rho = p = 0 between them."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    sl_tail = ul + 2.0 * cl / (g - 1.0)
    sr_tail = ur - 2.0 * cr / (g - 1.0)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    rho = np.zeros_like(xi)
    u = np.zeros_like(xi)
    p = np.zeros_like(xi)
    for n, s in enumerate(xi):
        if s <= ul - cl:
            rho[n], u[n], p[n] = rl, ul, pl
        elif s < sl_tail:
            c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
            rho[n] = rl * (c / cl) ** (2.0 / (g - 1.0))
            u[n] = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
            p[n] = pl * (c / cl) ** (2.0 * g / (g - 1.0))
        elif s <= sr_tail:
            rho[n], u[n], p[n] = 0.0, s, 0.0
        elif s < ur + cr:
            c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
            rho[n] = rr * (c / cr) ** (2.0 / (g - 1.0))
            u[n] = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
            p[n] = pr * (c / cr) ** (2.0 * g / (g - 1.0))
        else:
            rho[n], u[n], p[n] = rr, ur, pr
    return rho, u, p


def sample(left, right, xi, g=GAMMA):
    """(rho, u, p) arrays of the exact solution at similarity coordinates xi = (x - x0)/t."""
    if vacuum_forms(left, right, g):
        return _sample_vacuum(left, right, xi, g)
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    xi = np.atleast_1d(np.asarray(xi, dtype=np.float64))
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for n, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                rsl = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                rho[n], u[n], p[n] = (rl, ul, pl) if s <= sl else (rsl, us, ps)
            else:  # left rarefaction
                rsl = rl * (ps / pl) ** (1.0 / g)
                csl = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                shl, stl = ul - cl, us - csl
                if s <= shl:
                    rho[n], u[n], p[n] = rl, ul, pl
                elif s >= stl:
                    rho[n], u[n], p[n] = rsl, us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * (ul - s))
                    uu = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    rr_ = rl * (c / cl) ** (2.0 / (g - 1.0))
                    rho[n], u[n], p[n] = rr_, uu, pl * (c / cl) ** (2.0 * g / (g - 1.0))
        else:  # right of the contact
            if ps > pr:  # right shock
                rsr = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                rho[n], u[n], p[n] = (rsr, us, ps) if s <= sr else (rr, ur, pr)
            else:  # right rarefaction
                rsr = rr * (ps / pr) ** (1.0 / g)
                csr = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                shr, stt = ur + cr, us + csr
                if s >= shr:
                    rho[n], u[n], p[n] = rr, ur, pr
                elif s <= stt:
                    rho[n], u[n], p[n] = rsr, us, ps
                else:
                    c = 2.0 / (g + 1.0) * (cr - 0.5 * (g - 1.0) * (ur - s))
                    uu = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    rr_ = rr * (c / cr) ** (2.0 / (g - 1.0))
                    rho[n], u[n], p[n] = rr_, uu, pr * (c / cr) ** (2.0 * g / (g - 1.0))
    return rho, u, p


def wave_positions(left, right, g=GAMMA):
    """Speeds of the wave edges: dict with keys for the left wave, contact and right wave."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    out = {"contact": us, "p_star": ps}
    if ps > pl:
        out["left_shock"] = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
    else:
        out["left_head"] = ul - cl
        out["left_tail"] = us - cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
    if ps > pr:
        out["right_shock"] = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
    else:
        out["right_head"] = ur + cr
        out["right_tail"] = us + cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
    return out
