"""Extended-precision restatement of one FDLBM time step (test infrastructure only).

This is a second, independent reading of the scheme of Gan et al. (arXiv 0801.4169),
written in mpmath at a chosen number of decimal digits. It shares no code with the
FP64 C oracle (fdlbm_oracle.c) and none with the CUDA library. Its purpose is to tell,
for a run that the FP64 oracle rejects (a node reaching T <= 0 or n <= 0 within a few
steps), whether the scheme itself produces that state in exact arithmetic, or whether
it is FP64 cancellation: at high Mach number the equilibrium of Eq. 10 has values of
size kappa * n with kappa = sum |f_eq| / n up to 1e12, so an FP64 rounding can move a
moment by kappa * 1e-16 * n.

What it computes, in the paper's order, at every step:
  1. moments n, u, T of Eqs. 3-5 at every interior node and at the ghost node next
     to each edge (the ghost macros are those of the ghost f);
  2. at every interior node: F_k(theta) and F_0 (Eqs. 11-13), f_eq (Eq. 10, all five
     terms inside nF_k[...]), kappa_alpha (Eq. 15) and the switch theta_alphaI
     (Eq. 16) from P = nT at I-1, I, I+1 along alpha;
  3. Eq. 17 for every velocity, its alpha = x, y terms added, the relaxation term
     once;
  4. the ghost ring (width 2) of the new field from the boundary kinds.

Inputs: the model's speeds (1, 1.92, 2.99, 4.49), dx, dy, dt, tau, lambda and the
initial macros are the binary64 numbers the FP64 oracle and the library use,
converted exactly; the direction cosines (0, +-1, +-sqrt(1/2)) and everything after
are carried at `dps` digits. Boundary kinds and their mechanics are those of the
library (the paper names them, Sec. 5.2, but gives no mechanics): periodic wrap;
outflow copies the edge node into both ghost layers; Dirichlet ghosts hold f_eq of
the side's state; a specular wall mirrors node -1-j onto node j with the normal
velocity reversed. The x-ghost columns of interior rows are filled first, then the
y-ghost rows over the whole padded width.

It is slow (a few milliseconds per node and step at 40 digits): it is meant for the
first steps of small grids or windows.
"""
import mpmath as mp
import numpy as np

Q = 33
NG = 2
PERIODIC, OUTFLOW, DIRICHLET, WALL = 0, 1, 2, 3
NO_LW, NO_DISP, NO_VISC, SWITCH_CONST = 1, 2, 4, 8
SPEEDS = (1.0, 1.92, 2.99, 4.49)


def _vel_table():
    """(vx, vy, ring) per q: q = 0 rest; q = 1 + 8(k-1) + (i-1) has speed v_k and the
    direction at angle i*pi/4 (Eq. 1)."""
    h = mp.sqrt(mp.mpf(1) / 2)
    one, zero = mp.mpf(1), mp.mpf(0)
    cosines = {1: (h, h), 2: (zero, one), 3: (-h, h), 4: (-one, zero),
               5: (-h, -h), 6: (zero, -one), 7: (h, -h), 8: (one, zero)}
    vx, vy, ring = [zero], [zero], [0]
    for k in range(1, 5):
        v = mp.mpf(SPEEDS[k - 1])
        for i in range(1, 9):
            cx, cy = cosines[i]
            vx.append(v * cx)
            vy.append(v * cy)
            ring.append(k)
    return vx, vy, ring


def weights(theta):
    """(F_0, F_1..F_4) of Eqs. 11-13 at theta (mp numbers)."""
    v2 = [None] + [mp.mpf(s) ** 2 for s in SPEEDS]

    def nxt(k, l):  # cyclic index {k+l} of Eq. 13
        return k + l if k + l <= 4 else k + l - 4

    F = [None] * 5
    for k in range(1, 5):
        a, b, c = v2[nxt(k, 1)], v2[nxt(k, 2)], v2[nxt(k, 3)]
        den = v2[k] * (v2[k] - a) * (v2[k] - b) * (v2[k] - c)
        num = 48 * theta ** 4 - 6 * (a + b + c) * theta ** 3 + (a * b + b * c + c * a) * theta ** 2 \
            - a * b * c / 4 * theta
        F[k] = num / den
    F[0] = 1 - 8 * (F[1] + F[2] + F[3] + F[4])
    return F


def feq(n, ux, uy, T, table):
    """The 33 values of Eq. 10 (m = 1, theta = T), as mp numbers."""
    vx, vy, ring = table
    th = T
    F = weights(th)
    u2 = ux * ux + uy * uy
    g = 1 - u2 / (2 * th)
    out = []
    for q in range(Q):
        s = (vx[q] * ux + vy[q] * uy) / th  # v.u / theta
        br = (1 - u2 / (2 * th) + u2 * u2 / (8 * th * th)) + s * g + s * s / 2 * g + s ** 3 / 6 + s ** 4 / 24
        out.append(n * F[ring[q]] * br)
    return out


def moments(fs, table):
    """(n, ux, uy, T) of Eqs. 3-5 from one node's 33 values."""
    vx, vy, _ = table
    n = mp.fsum(fs)
    jx = mp.fsum(vx[q] * fs[q] for q in range(Q))
    jy = mp.fsum(vy[q] * fs[q] for q in range(Q))
    ux, uy = jx / n, jy / n
    P = mp.fsum(((vx[q] - ux) ** 2 + (vy[q] - uy) ** 2) / 2 * fs[q] for q in range(Q))
    return n, ux, uy, P / n


class MPSim:
    """An nx x ny solve at `dps` decimal digits (small grids: a few ms per node and step)."""

    def __init__(self, nx, ny, dx, dy, dt, tau, lam, bc, bstate=None, flags=0, dps=40):
        self.nx, self.ny, self.dps = int(nx), int(ny), int(dps)
        self.bc = tuple(int(b) for b in bc)
        self.flags = int(flags)
        with mp.workdps(self.dps):
            self.table = _vel_table()
            self.dx, self.dy, self.dt, self.tau, self.lam = (mp.mpf(float(a)) for a in (dx, dy, dt, tau, lam))
            bs = np.zeros((4, 4)) if bstate is None else np.asarray(bstate, dtype=np.float64)
            self.bfeq = [feq(*[mp.mpf(float(a)) for a in bs[s]], self.table) if self.bc[s] == DIRICHLET else None
                         for s in range(4)]
        # f[q][row][col], row = j + 2, col = i + 2
        self.f = None
        self.steps_done = 0

    # --- mirrors of a direction at a wall (y-wall: angle -> -angle; x-wall: angle -> pi - angle)
    @staticmethod
    def _mirror(q, axis):
        if q == 0:
            return 0
        k, i = 1 + (q - 1) // 8, 1 + (q - 1) % 8
        j = (8 - i) % 8 if axis == 1 else (4 - i) % 8
        if j == 0:
            j = 8
        return 1 + 8 * (k - 1) + (j - 1)

    def _fill_ghosts(self, f):
        nx, ny = self.nx, self.ny
        L, R, B, T = self.bc

        def src_x(c, side):
            kind = L if side == 0 else R
            if kind == PERIODIC:
                return c % nx
            if kind == OUTFLOW:
                return 0 if side == 0 else nx - 1
            if kind == WALL:
                return -1 - c if side == 0 else 2 * nx - 1 - c
            return None

        def src_y(c, side):
            kind = B if side == 2 else T
            if kind == PERIODIC:
                return c % ny
            if kind == OUTFLOW:
                return 0 if side == 2 else ny - 1
            if kind == WALL:
                return -1 - c if side == 2 else 2 * ny - 1 - c
            return None

        for j in range(ny):
            for c, side in ((-2, 0), (-1, 0), (nx, 1), (nx + 1, 1)):
                kind = self.bc[side]
                for q in range(Q):
                    if kind == DIRICHLET:
                        val = self.bfeq[side][q]
                    else:
                        s = src_x(c, side)
                        qq = self._mirror(q, 0) if kind == WALL else q
                        val = f[qq][j + NG][s + NG]
                    f[q][j + NG][c + NG] = val
        for i in range(-NG, nx + NG):
            for c, side in ((-2, 2), (-1, 2), (ny, 3), (ny + 1, 3)):
                kind = self.bc[side]
                for q in range(Q):
                    if kind == DIRICHLET:
                        val = self.bfeq[side][q]
                    else:
                        s = src_y(c, side)
                        qq = self._mirror(q, 1) if kind == WALL else q
                        val = f[qq][s + NG][i + NG]
                    f[q][c + NG][i + NG] = val

    def set_macro(self, rho, u, v, T):
        """f = f_eq of the given FP64 macros (ny x nx arrays, converted exactly)."""
        arrs = [np.broadcast_to(np.asarray(a, dtype=np.float64), (self.ny, self.nx)) for a in (rho, u, v, T)]
        with mp.workdps(self.dps):
            zero = mp.mpf(0)
            f = [[[zero] * (self.nx + 2 * NG) for _ in range(self.ny + 2 * NG)] for _ in range(Q)]
            for j in range(self.ny):
                for i in range(self.nx):
                    fe = feq(*[mp.mpf(float(a[j, i])) for a in arrs], self.table)
                    for q in range(Q):
                        f[q][j + NG][i + NG] = fe[q]
            self._fill_ghosts(f)
        self.f = f
        self.steps_done = 0

    def _node(self, f, i, j):
        return [f[q][j + NG][i + NG] for q in range(Q)]

    def macros(self):
        """(n, ux, uy, T) of the interior as ny x nx arrays of mp numbers."""
        with mp.workdps(self.dps):
            out = [np.empty((self.ny, self.nx), dtype=object) for _ in range(4)]
            for j in range(self.ny):
                for i in range(self.nx):
                    m = moments(self._node(self.f, i, j), self.table)
                    for a in range(4):
                        out[a][j, i] = m[a]
        return out

    def step(self, nsteps=1):
        """Advance; returns 0, or -4 when a needed node has n <= 0 or T <= 0 at a step's start."""
        for _ in range(int(nsteps)):
            rc = self._step_once()
            if rc:
                return rc
        return 0

    def _step_once(self):
        nx, ny, f = self.nx, self.ny, self.f
        vx, vy, _ = self.table
        with mp.workdps(self.dps):
            mom = {}
            for j in range(-1, ny + 1):
                for i in range(-1, nx + 1):
                    inx, iny = 0 <= i < nx, 0 <= j < ny
                    if not ((inx and iny) or (iny and i in (-1, nx)) or (inx and j in (-1, ny))):
                        continue
                    m = moments(self._node(f, i, j), self.table)
                    if not (m[0] > 0 and m[3] > 0):
                        return -4
                    mom[(i, j)] = m
            r = self.dt / self.tau
            dr = (self.dx, self.dy)
            zero = mp.mpf(0)
            fn = [[[zero] * (nx + 2 * NG) for _ in range(ny + 2 * NG)] for _ in range(Q)]
            for j in range(ny):
                for i in range(nx):
                    n, ux, uy, T = mom[(i, j)]
                    fe = feq(n, ux, uy, T, self.table)
                    nu = []
                    for a, (di, dj) in enumerate(((1, 0), (0, 1))):
                        Pp = mom[(i + di, j + dj)][0] * mom[(i + di, j + dj)][3]
                        P0 = n * T
                        Pm = mom[(i - di, j - dj)][0] * mom[(i - di, j - dj)][3]
                        th = self.lam if self.flags & SWITCH_CONST else self.lam * abs((Pp - 2 * P0 + Pm) / (Pp + 2 * P0 + Pm))
                        kap = abs((ux if a == 0 else uy) * self.dt / dr[a])
                        nu.append(th * kap * (1 - kap) / 2)
                    for q in range(Q):
                        c0 = f[q][j + NG][i + NG]
                        new = c0 - r * (c0 - fe[q])
                        for a, (di, dj) in enumerate(((1, 0), (0, 1))):
                            p1 = f[q][j + NG + dj][i + NG + di]
                            m1 = f[q][j + NG - dj][i + NG - di]
                            p2 = f[q][j + NG + 2 * dj][i + NG + 2 * di]
                            m2 = f[q][j + NG - 2 * dj][i + NG - 2 * di]
                            c = (vx[q] if a == 0 else vy[q]) * self.dt / dr[a]  # Eq. 15
                            new -= c / 2 * (p1 - m1)                                       # line I
                            if not self.flags & NO_LW:
                                new += c * c / 2 * (p1 - 2 * c0 + m1)                      # line II
                            if not self.flags & NO_DISP:
                                new += c * (1 - c * c) / 12 * (p2 - 2 * p1 + 2 * m1 - m2)   # line III
                            if not self.flags & NO_VISC:
                                new += nu[a] * (p1 - 2 * c0 + m1)                          # line IV
                        fn[q][j + NG][i + NG] = new
            self._fill_ghosts(fn)
        self.f = fn
        self.steps_done += 1
        return 0
