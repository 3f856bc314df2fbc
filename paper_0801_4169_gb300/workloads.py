"""Seeded synthetic workloads (initial and boundary data) for the FDLBM solver.

This module only builds inputs: grids, parameters and the macroscopic fields
(rho, u, v, T) a run starts from. It holds none of the scheme's arithmetic,
and both the CUDA path and the CPU oracle read their inputs from it. Shock
states use the textbook Rankine-Hugoniot jump for an ideal gas with the
model's gamma = 2 (2-D, e_int = nT). Sec. 5.2 of the paper prints two such
states (Eqs. 26, 27); the tests check this module against them.

Workloads (all FP64 macros, x fastest, m = 1 so rho = n and p = rho*T):
  sod           Sod tube of Sec. 5.1 (Eq. 21): 400 x 4, dx = 1e-3, dt = tau = 1e-5,
                lambda = 2, outflow in x, periodic in y, 2000 steps.
  shock_tube    strong normal shock: Mach Ms relative to the upstream gas
                (rho1 = 1, T1 = 0.5), upstream flowing into the shock at -U.
                4000 x 4 by default, lambda = 2, 5000 steps. The defaults
                (Ms = 10, U = 6) are the strongest shock the scheme carries.
                Ms = 20 into gas at rest is rejected after one step by the
                scheme (non-positive temperature for every lambda tried).
  reflection    steady regular reflection of Sec. 5.2 (Eq. 26): Mach-20 stream
                (1, 20, 0, 0.5) entering on the left, top state (50/17, 16.7,
                -5.71578, 22.61); Dirichlet left and top, outflow right, specular
                wall at the bottom; lambda = 20, dt = tau = 0.0025 dx. The paper gives no initial field;
                the domain starts in the top state and the incident shock forms at
                the top-left corner (init="shock" starts from a sharp 30-degree shock, which
                the scheme rejects within a few steps for lambda = 1 and 5 but runs at 20).
  riemann4q     four-quadrant 2-D Riemann problem with seeded quadrant states,
                outflow on every side.
  serving_requests  seeded Poisson stream of shock-tube solves of mixed size,
                Mach number, length and precision.
  riemann1d     the 1-D Riemann problems of Sec. 5.1 (Eqs. 21-25) on ny = 1.
  dmr           double Mach reflection of Sec. 5.2.2 (Eq. 27): 60-degree shock into gas at rest,
                wall from x = 0.08, a moving Dirichlet segment on the top boundary.
  vn_sec4       the von Neumann sweeps of Sec. 4 (Figs. 2, 4, 5, 6): uniform states,
                lambda and scheme variants, each over nk wave numbers k dx in (0, pi].
"""
import math
from dataclasses import dataclass, field

import numpy as np

PERIODIC, OUTFLOW, DIRICHLET, WALL = 0, 1, 2, 3
GAMMA = 2.0


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    tau: float
    lam: float
    bc: tuple
    steps: int
    rho: np.ndarray
    u: np.ndarray
    v: np.ndarray
    T: np.ndarray
    bstate: np.ndarray = field(default_factory=lambda: np.zeros((4, 4)))
    meta: dict = field(default_factory=dict)

    @property
    def sites(self):
        return self.nx * self.ny

    def macros(self):
        return self.rho, self.u, self.v, self.T


def _fields(nx, ny, fill):
    return [np.ascontiguousarray(np.broadcast_to(np.asarray(a, dtype=np.float64), (ny, nx)))
            for a in fill]


def rh_moving_shock(Ms, rho1=1.0, T1=1.0, u1=0.0, g=GAMMA):
    """Gas behind a normal shock moving in +x at Mach Ms relative to upstream gas (rho1, u1, T1).

    Returns (rho2, u2, T2, W_lab)."""
    p1 = rho1 * T1
    c1 = math.sqrt(g * p1 / rho1)
    m2 = Ms * Ms
    rr = (g + 1.0) * m2 / ((g - 1.0) * m2 + 2.0)
    pr = (2.0 * g * m2 - (g - 1.0)) / (g + 1.0)
    W = Ms * c1
    return rho1 * rr, u1 + W * (1.0 - 1.0 / rr), T1 * pr / rr, u1 + W


def sod(nx=400, ny=4, steps=2000, dx=1e-3, dt=1e-5, tau=1e-5, lam=2.0):
    """Sod shock tube (Eq. 21): left (1, 0, 0, 1), right (0.125, 0, 0, 0.8), split at 0.5 L."""
    x = (np.arange(nx) + 0.5) * dx
    left = (x < 0.5 * nx * dx)[None, :]
    rho, u, v, T = _fields(nx, ny, (np.where(left, 1.0, 0.125), 0.0, 0.0, np.where(left, 1.0, 0.8)))
    return Workload("sod%dx%d" % (nx, ny), nx, ny, dx, dx, dt, tau, lam,
                    (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC), steps, rho, u, v, T,
                    meta=dict(left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), x0=0.5 * nx * dx))


def shock_tube(nx=4000, ny=4, steps=5000, Ms=10.0, U=6.0, T1=0.5, rho1=1.0, dx=1e-3, dt=1e-5,
               tau=1e-5, lam=2.0, x0_frac=0.1):
    """Normal shock of Mach Ms (relative to the upstream gas) at x0 = x0_frac * L moving in +x.

    Upstream gas (rho1, -U, 0, T1) flows into the shock; the post-shock state is the
    Rankine-Hugoniot state (gamma = 2)."""
    c1 = math.sqrt(GAMMA * T1)
    rho2, u2, T2, W = rh_moving_shock(Ms, rho1, T1, -U * c1)
    x = (np.arange(nx) + 0.5) * dx
    x0 = x0_frac * nx * dx
    post = (x < x0)[None, :]
    rho, u, v, T = _fields(nx, ny, (np.where(post, rho2, rho1), np.where(post, u2, -U * c1), 0.0,
                                    np.where(post, T2, T1)))
    return Workload("shock%gx%dx%d" % (Ms, nx, ny), nx, ny, dx, dx, dt, tau, lam,
                    (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC), steps, rho, u, v, T,
                    meta=dict(Ms=Ms, U=U, post=(rho2, u2, 0.0, T2), pre=(rho1, -U * c1, 0.0, T1),
                              W_lab=W, x0=x0))


REFLECTION_PRE = (1.0, 20.0, 0.0, 0.5)             # Eq. 26, left boundary
REFLECTION_POST = (50.0 / 17.0, 16.7, -5.71578, 22.61)  # Eq. 26, top boundary


def reflection(nx=1200, ny=300, dx=None, height=0.3, steps=10000, dt=None, tau=None, lam=20.0, init="post"):
    """Steady regular reflection (Sec. 5.2, Eq. 26) on an nx x ny grid of height 0.3.

    dt = tau = 0.0025 dx by default, so kappa_x = u dt/dx = 0.05 in the Mach-20 stream at every
    resolution (2.5e-6 at dx = 1e-3; dt = 1e-5 there fails within 1000 steps for lambda up to 20).
    init="post": the whole domain starts in the top (post-shock) state; init="shock": post-shock
    above the incident-shock line y = height - x tan 30 deg, pre-shock below it."""
    if dx is None:
        dx = height / ny
    if dt is None:
        dt = 0.0025 * dx
    if tau is None:
        tau = dt
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    if init == "post":
        above = np.ones((ny, nx), dtype=bool)
    else:
        above = Y > height - X * math.tan(math.radians(30.0))
    rho, u, v, T = _fields(nx, ny, [np.where(above, REFLECTION_POST[i], REFLECTION_PRE[i]) for i in range(4)])
    bstate = np.zeros((4, 4))
    bstate[0] = REFLECTION_PRE
    bstate[3] = REFLECTION_POST
    return Workload("reflection%dx%d" % (nx, ny), nx, ny, dx, dx, dt, tau, lam,
                    (DIRICHLET, OUTFLOW, WALL, DIRICHLET), steps, rho, u, v, T, bstate=bstate,
                    meta=dict(pre=REFLECTION_PRE, post=REFLECTION_POST, height=height))


def riemann4q(n=4096, seed=0, steps=2000, dx=2.5e-4, dt=2.5e-6, tau=2.5e-6, lam=3.0, mach_max=1.0,
              ny=None, rho_range=(0.5, 2.0), p_range=(0.5, 1.5)):
    """Four-quadrant 2-D Riemann problem with quadrant states drawn from a PCG64 stream.

    Per quadrant: rho ~ U[rho_range], p ~ U[p_range], T = p / rho, Mach ~ U[0, mach_max],
    direction ~ U[0, 2 pi), (u, v) = Mach * sqrt(2 T) * (cos, sin). Split at (nx/2, ny/2).
    The defaults (rho in [0.5, 2], p in [0.5, 1.5], Mach <= 1, lambda = 3) keep seeds 0-2 finite
    for 2000 steps; wider ranges (p down to 0.03, Mach up to 10) are rejected by the scheme within
    the first steps for some seeds."""
    nx = n
    ny = n if ny is None else ny
    rng = np.random.Generator(np.random.PCG64(seed))
    states = []
    for _ in range(4):
        rho = rng.uniform(*rho_range)
        p = rng.uniform(*p_range)
        T = p / rho
        M = rng.uniform(0.0, mach_max)
        phi = rng.uniform(0.0, 2.0 * math.pi)
        c = math.sqrt(GAMMA * T)
        states.append((rho, M * c * math.cos(phi), M * c * math.sin(phi), T))
    ix = (np.arange(nx) >= nx // 2)[None, :]
    iy = (np.arange(ny) >= ny // 2)[:, None]
    quad = (ix.astype(int) + 2 * iy.astype(int))  # 0: SW, 1: SE, 2: NW, 3: NE
    arr = np.array(states)
    rho, u, v, T = _fields(nx, ny, [arr[quad, i] for i in range(4)])
    return Workload("riemann4q%dx%d_s%d" % (nx, ny, seed), nx, ny, dx, dx, dt, tau, lam,
                    (OUTFLOW,) * 4, steps, rho, u, v, T, meta=dict(states=states, seed=seed))


DMR_PRE = (2.0, 0.0, 0.0, 0.5)  # Eq. 27, gas ahead of the shock (sound speed 1)


def dmr(Ms=20.0, nx=500, ny=200, dx=1e-3, dt=1e-5, tau=None, lam=20.0, steps=750, x_wall=0.08):
    """Double Mach reflection (Sec. 5.2.2, Eq. 27) on an nx x ny grid of spacing dx.

    A planar shock of normal Mach Ms runs into gas at rest (2, 0, 0, 0.5) at 60 degrees to the x axis;
    behind it the gamma = 2 Rankine-Hugoniot state (400/67, 13.3, 89.2775 at Ms = 20) moves along the
    shock normal (cos 30, -sin 30). The shock line is y = h(x, t) = sqrt(3) (x - x_wall) - 2 W t
    (W = Ms c1, so 2W = 40 at Ms = 20), post-shock gas above it. Boundaries: Dirichlet post-shock
    state on the left; outflow on the right; at the bottom a specular wall from x = x_wall on, the
    post-shock state before it; at the top the post-shock state for x below
    g(t) = x_wall + (H + 2 W t)/sqrt(3) (H the domain height) and the gas at rest beyond. The two
    segments are returned in meta["segments"] as (side, c0, speed, lower, state). The scheme
    rejects Ms = 20 (the Eq. 27 data) in exact arithmetic; the default Ms is the paper's."""
    if tau is None:
        tau = dt
    rho1, u1, v1, T1 = DMR_PRE
    rho2, un, T2, W = rh_moving_shock(Ms, rho1, T1)
    c30, s30 = math.cos(math.radians(30.0)), math.sin(math.radians(30.0))
    post = (rho2, un * c30, -un * s30, T2)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dx
    X, Y = np.meshgrid(x, y)
    behind = Y >= math.sqrt(3.0) * (X - x_wall)
    rho, u, v, T = _fields(nx, ny, [np.where(behind, post[i], DMR_PRE[i]) for i in range(4)])
    H = ny * dx
    bstate = np.zeros((4, 4))
    bstate[0] = post   # left: Dirichlet post-shock
    bstate[3] = DMR_PRE  # top beyond the moving segment
    segments = [(2, x_wall, 0.0, True, post),                                   # bottom, before the wall
                (3, x_wall + H / math.sqrt(3.0), 2.0 * W / math.sqrt(3.0), True, post)]  # top, moving
    return Workload("dmr%gx%dx%d" % (Ms, nx, ny), nx, ny, dx, dx, dt, tau, lam,
                    (DIRICHLET, OUTFLOW, WALL, DIRICHLET), steps, rho, u, v, T, bstate=bstate,
                    meta=dict(pre=DMR_PRE, post=post, W=W, x_wall=x_wall, segments=segments, Ms=Ms))


RIEMANN1D = {
    # name: (left (rho,u,v,T), right, dx, dt, tau, lambda, t_end)   (Sec. 5.1, Eqs. 21-25)
    "sod": ((1.0, 0.0, 0.0, 1.0), (0.125, 0.0, 0.0, 0.8), 1e-3, 1e-5, 1e-4, 2.0, 0.2),
    "lax": ((0.445, 0.698, 0.0, 7.928), (0.5, 0.0, 0.0, 1.142), 1e-3, 1e-5, 1e-4, 1.0, 0.2),
    "sjogreen": ((1.0, -2.0, 0.0, 0.4), (1.0, 2.0, 0.0, 0.4), 3e-3, 1e-5, 1e-5, 1.8, 0.018),
    "colella": ((1.0, 0.0, 0.0, 1000.0), (1.0, 0.0, 0.0, 0.01), 3e-3, 1e-5, 1e-5, 20.0, 0.05),
    "collision": ((5.99924, 19.5975, 0.0, 76.8254), (5.99242, -6.19633, 0.0, 7.69222), 2e-3, 1e-5, 1e-5,
                  1.0, 0.12),
    # Sec. 4, Fig. 3: the dispersion on/off tube, "otherwise as Fig. 2" (dx = 3e-3, dt = tau = 1e-5).
    # The paper gives no end time; 0.03 keeps both shocks inside 400 nodes.
    "fig3": ((10.0, 10.0, 0.0, 5.0), (10.0, 0.0, 0.0, 5.0), 3e-3, 1e-5, 1e-5, 2.0, 0.03),
}


def riemann1d(name, nx=1000, ny=1, steps=None):
    """One of the Sec. 5.1 Riemann problems on nx nodes split at the middle (periodic y)."""
    L, R, dx, dt, tau, lam, tend = RIEMANN1D[name]
    if steps is None:
        steps = int(round(tend / dt))
    x = (np.arange(nx) + 0.5) * dx
    left = (x < 0.5 * nx * dx)[None, :]
    rho, u, v, T = _fields(nx, ny, [np.where(left, L[i], R[i]) for i in range(4)])
    return Workload("%s%d" % (name, nx), nx, ny, dx, dx, dt, tau, lam,
                    (OUTFLOW, OUTFLOW, PERIODIC, PERIODIC), steps, rho, u, v, T,
                    meta=dict(left=L, right=R, x0=0.5 * nx * dx))


@dataclass
class Request:
    rid: int
    arrival_s: float
    nx: int
    ny: int
    Ms: float
    steps: int
    prec: int  # 0 = FP64, 1 = FP32 storage


def serving_requests(n=512, seed=0, mean_gap_s=0.005, nx_range=(256, 16384), ms_range=(2.0, 10.0),
                     steps_range=(2000, 20000), ny=4):
    """Seeded Poisson arrivals (exponential gaps) of shock-tube solves.

    nx ~ U{nx_range}, Ms ~ U[ms_range], steps ~ U{steps_range}, precision ~ Bernoulli(1/2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(mean_gap_s)
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        Ms = float(rng.uniform(*ms_range))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        prec = int(rng.integers(0, 2))
        out.append(Request(i, t, nx, ny, Ms, steps, prec))
    return out


def request_workload(req, lam=2.0):
    """The shock-tube solve a serving request describes (upstream flowing at -(Ms - 2) c1)."""
    return shock_tube(nx=req.nx, ny=req.ny, steps=req.steps, Ms=req.Ms, U=max(0.0, req.Ms - 2.0), lam=lam)


# flags of the Sec. 4 scheme variants (values of enum fdlbm_flags)
_NO_LW, _NO_DISP, _NO_VISC = 1, 2, 4


def vn_sec4_curves():
    """The curves of Sec. 4 as (label, (rho, u1, u2, T), lambda, flags). All at dx = dy = 3e-3,
    dt = tau = 1e-5, speeds (1, 1.92, 2.99, 4.49), wave vector along x.

    Fig. 2: (2, 30, 0, 1), lambda = 0.5, Eq. 17 with line I only, lines I-II, lines I and III, all.
    Fig. 4: the same state, lambda in {0.05, 0.1, 0.5, 1, 1.8, 2, 3}.
    Fig. 5: u1 = 5, lambda = 0, T in {1, 5, 15, 25} (rho = 2 kept from Fig. 2).
    Fig. 6: lambda = 0, u1 from 0 to 30 (steps of 5), T = 1."""
    base = (2.0, 30.0, 0.0, 1.0)
    c = [("fig2 line I", base, 0.5, _NO_LW | _NO_DISP | _NO_VISC), ("fig2 lines I-II", base, 0.5, _NO_DISP | _NO_VISC),
         ("fig2 lines I,III", base, 0.5, _NO_LW | _NO_VISC), ("fig2 all", base, 0.5, 0)]
    c += [("fig4 lambda=%g" % l, base, l, 0) for l in (0.05, 0.1, 0.5, 1.0, 1.8, 2.0, 3.0)]
    c += [("fig5 T=%g" % T, (2.0, 5.0, 0.0, float(T)), 0.0, 0) for T in (1, 5, 15, 25)]
    c += [("fig6 u1=%g" % u, (2.0, float(u), 0.0, 1.0), 0.0, 0) for u in (0, 5, 10, 15, 20, 25, 30)]
    return c


VN_SEC4_GRID = (3e-3, 3e-3, 1e-5, 1e-5)  # dx, dy, dt, tau


def vn_sec4_cases(nk=256):
    """(records, curves, xi): one case per (curve, k dx), curve-major, as plain numbers
    [rho, u1, u2, T, xi_x, xi_y, lambda, flags] (n, 8)."""
    curves = vn_sec4_curves()
    xi = np.linspace(np.pi / nk, np.pi, nk)
    rows = []
    for _, st, lam, fl in curves:
        for x in xi:
            rows.append([st[0], st[1], st[2], st[3], x, 0.0, lam, fl])
    return np.array(rows), curves, xi
