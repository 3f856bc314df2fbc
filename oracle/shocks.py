"""Rankine-Hugoniot and oblique-shock relations for gamma = 2 (test infrastructure only).

Used to check the shock states the paper prints for its reflection tests
(Sec. 5.2: the Eq. 26 top state behind the incident shock of a Mach-20
stream at 30 degrees; the Eq. 27 post-shock state of a shock-Mach-20 wave in the
double-Mach set-up) and the plateaus of the strong shock tube. Written from the conservation of mass, momentum and energy
across a steady discontinuity for an ideal gas with p = rho T (m = 1).
"""
import math

GAMMA = 2.0


def normal_shock(Ms, rho1=1.0, p1=1.0, g=GAMMA):
    """Moving normal shock of Mach Ms into gas at rest (rho1, 0, p1).

    Returns dict(rho2, u2, p2, T2, W) with W the lab-frame shock speed and u2
    the lab-frame gas velocity behind the shock.
    """
    c1 = math.sqrt(g * p1 / rho1)
    M2 = Ms * Ms
    rho2 = rho1 * (g + 1.0) * M2 / ((g - 1.0) * M2 + 2.0)
    p2 = p1 * (2.0 * g * M2 - (g - 1.0)) / (g + 1.0)
    W = Ms * c1
    u2 = W * (1.0 - rho1 / rho2)
    return dict(rho2=rho2, u2=u2, p2=p2, T2=p2 / rho2, W=W, c1=c1)


def oblique_shock(M1, beta, g=GAMMA):
    """Steady oblique shock at wave angle beta (radians) in a stream of Mach M1.

    Returns dict(theta, rho_ratio, p_ratio, M2): flow deflection, density and
    pressure ratios, and the downstream Mach number.
    """
    Mn1 = M1 * math.sin(beta)
    rr = (g + 1.0) * Mn1 ** 2 / ((g - 1.0) * Mn1 ** 2 + 2.0)
    pr = (2.0 * g * Mn1 ** 2 - (g - 1.0)) / (g + 1.0)
    theta = math.atan(2.0 / math.tan(beta) * (M1 ** 2 * math.sin(beta) ** 2 - 1.0)
                      / (M1 ** 2 * (g + math.cos(2.0 * beta)) + 2.0))
    Mn2 = math.sqrt((1.0 + 0.5 * (g - 1.0) * Mn1 ** 2) / (g * Mn1 ** 2 - 0.5 * (g - 1.0)))
    M2 = Mn2 / math.sin(beta - theta)
    return dict(theta=theta, rho_ratio=rr, p_ratio=pr, M2=M2)


def weak_beta(M1, theta, g=GAMMA):
    """Weak-solution wave angle for deflection theta (radians) by bisection on the theta-beta-M relation."""
    mu = math.asin(1.0 / M1)
    # locate the maximum-deflection angle, then bisect on the weak branch [mu, beta_max]
    lo, hi = mu, 0.5 * math.pi
    for _ in range(200):
        m1 = lo + (hi - lo) / 3.0
        m2 = hi - (hi - lo) / 3.0
        if oblique_shock(M1, m1, g)["theta"] < oblique_shock(M1, m2, g)["theta"]:
            lo = m1
        else:
            hi = m2
    bmax = 0.5 * (lo + hi)
    if oblique_shock(M1, bmax, g)["theta"] < theta:
        raise ValueError("deflection exceeds the attached-shock maximum")
    a, b = mu + 1e-15, bmax
    for _ in range(200):
        m = 0.5 * (a + b)
        if oblique_shock(M1, m, g)["theta"] < theta:
            a = m
        else:
            b = m
    return 0.5 * (a + b)


def regular_reflection(M1, beta1, rho1=1.0, u1=1.0, T1=None, g=GAMMA):
    """Two-shock regular reflection off a wall parallel to the incoming stream.

    The incident shock makes angle beta1 with the wall (and the stream). Returns
    the deflection theta, the region-2 Mach number, the reflected-shock angle to
    the wall, and the region-2 state (rho, u, v, T) for an incoming stream
    (rho1, u1 along +x, T1) whose shock descends in +x towards the wall.
    """
    s1 = oblique_shock(M1, beta1, g)
    theta = s1["theta"]
    beta_r = weak_beta(s1["M2"], theta, g)
    out = dict(theta=theta, M2=s1["M2"], beta_reflected_rel_flow=beta_r,
               reflected_angle_to_wall=beta_r - theta)
    if T1 is not None:
        rho2 = rho1 * s1["rho_ratio"]
        p2 = rho1 * T1 * s1["p_ratio"]
        un1 = u1 * math.sin(beta1)
        ut = u1 * math.cos(beta1)
        un2 = un1 / s1["rho_ratio"]
        # shock line direction t = (cos b, -sin b); downstream normal n = (sin b, cos b)
        ux = ut * math.cos(beta1) + un2 * math.sin(beta1)
        uy = -ut * math.sin(beta1) + un2 * math.cos(beta1)
        out["state2"] = (rho2, ux, uy, p2 / rho2)
    return out
