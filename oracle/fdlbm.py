"""ctypes wrapper over the C oracle (test infrastructure only).

The C source ``fdlbm_oracle.c`` restates the scheme of Gan et al. (arXiv
0801.4169): velocity set (Sec. 2, Eq. 1), moments (Eqs. 3-5), weights and
equilibrium (Eqs. 10-13), and the modified Lax-Wendroff step with dispersion
and artificial viscosity (Sec. 3, Eqs. 15-17). This module only marshals
arguments; all arithmetic is in the C file.
"""
import ctypes
import os

import numpy as np

from . import build as _build

Q = 33

# boundary kinds (left, right, bottom, top); HALO: ghosts written by the caller (a neighbouring
# sub-domain), never by the oracle's fill
PERIODIC, OUTFLOW, DIRICHLET, WALL, HALO = 0, 1, 2, 3, 4

# Eq. 17 variants (Sec. 4): drop line II, III, IV, or hold the switch at lambda
NO_LW, NO_DISP, NO_VISC, SWITCH_CONST = 1, 2, 4, 8

_lib = None


def lib():
    global _lib
    if _lib is None:
        # FDLBM_ORACLE_LIB lets the mutation tests load a deliberately broken copy
        path = os.environ.get("FDLBM_ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_velocities.argtypes = [dp, dp]
        L.orc_weights.argtypes = [ctypes.c_double, dp]
        L.orc_feq.argtypes = [ctypes.c_double] * 4 + [dp]
        L.orc_moments.argtypes = [dp, dp, dp, dp, dp]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 + [
            ctypes.POINTER(ctypes.c_int), dp, ctypes.c_int]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_macro.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_get_macro.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_set_f.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_f.argtypes = [ctypes.c_void_p, dp]
        L.orc_get_f_padded.argtypes = [ctypes.c_void_p, dp]
        L.orc_set_f_padded.argtypes = [ctypes.c_void_p, dp]
        L.orc_step.restype = ctypes.c_int
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.orc_set_segment.restype = ctypes.c_int
        L.orc_set_segment.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, dp]
        L.orc_steps_done.restype = ctypes.c_long
        L.orc_steps_done.argtypes = [ctypes.c_void_p]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def velocities():
    """(vx, vy), each shape (33,): Eq. 1 with speeds (1, 1.92, 2.99, 4.49)."""
    vx = np.zeros(Q)
    vy = np.zeros(Q)
    lib().orc_velocities(_p(vx), _p(vy))
    return vx, vy


def weights(theta):
    """(F_0, F_1..F_4) of Eqs. 11-12."""
    F = np.zeros(5)
    lib().orc_weights(float(theta), _p(F))
    return F


def feq(n, ux, uy, T):
    """f^eq (33,) of Eq. 10."""
    out = np.zeros(Q)
    lib().orc_feq(float(n), float(ux), float(uy), float(T), _p(out))
    return out


def moments(f):
    """(n, ux, uy, T) of Eqs. 3-5 from one site's 33 values."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = [ctypes.c_double() for _ in range(4)]
    lib().orc_moments(_p(f), *[ctypes.byref(o) for o in out])
    return tuple(o.value for o in out)


class Sim:
    """One FDLBM solve on an nx x ny grid with a width-2 ghost ring.

    bc = (left, right, bottom, top) in {PERIODIC, OUTFLOW, DIRICHLET, WALL};
    bstate[side] = (rho, u, v, T) for DIRICHLET sides.
    """

    def __init__(self, nx, ny, dx, dy, dt, tau, lam, bc, bstate=None, flags=0):
        self.nx, self.ny = int(nx), int(ny)
        bc_arr = (ctypes.c_int * 4)(*[int(b) for b in bc])
        bs = np.zeros((4, 4)) if bstate is None else np.ascontiguousarray(bstate, dtype=np.float64)
        self._bs = bs
        self._h = lib().orc_create(self.nx, self.ny, float(dx), float(dy), float(dt), float(tau),
                                   float(lam), bc_arr, _p(bs), int(flags))
        if not self._h:
            raise ValueError("orc_create rejected the arguments")

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def set_macro(self, rho, u, v, T):
        arrs = [np.ascontiguousarray(np.broadcast_to(a, (self.ny, self.nx)), dtype=np.float64)
                for a in (rho, u, v, T)]
        lib().orc_set_macro(self._h, *[_p(a) for a in arrs])

    def get_macro(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        lib().orc_get_macro(self._h, *[_p(a) for a in out])
        return tuple(out)

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(Q, self.ny, self.nx)
        lib().orc_set_f(self._h, _p(f))

    def get_f(self):
        f = np.zeros((Q, self.ny, self.nx))
        lib().orc_get_f(self._h, _p(f))
        return f

    def get_f_padded(self):
        f = np.zeros((Q, self.ny + 4, self.nx + 4))
        lib().orc_get_f_padded(self._h, _p(f))
        return f

    def set_segment(self, side, c0, speed, lower, state):
        """A Dirichlet segment on `side` (Sec. 5.2.2): the side's ghosts whose coordinate along it,
        (i + 1/2) dx or (j + 1/2) dy, is below (lower) or at/above (not lower) c0 + speed * t hold
        f_eq(state) at time t = steps * dt; the rest of the side keeps its kind. Set it before
        set_macro / set_f."""
        st = np.ascontiguousarray(state, dtype=np.float64)
        if lib().orc_set_segment(self._h, int(side), float(c0), float(speed), int(bool(lower)), _p(st)):
            raise ValueError("side out of range")

    def set_f_padded(self, f):
        """Write the whole padded buffer, ghosts included, as given (no ghost fill)."""
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(Q, self.ny + 4, self.nx + 4)
        lib().orc_set_f_padded(self._h, _p(f))

    def step(self, nsteps=1):
        """Advance nsteps; returns 0, or -4 if non-finite moments or P <= 0 appeared."""
        return int(lib().orc_step(self._h, int(nsteps)))

    @property
    def steps_done(self):
        return int(lib().orc_steps_done(self._h))
