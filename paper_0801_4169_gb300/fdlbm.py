"""Thin ctypes binding of the C ABI in include/fdlbm.h (libfdlbm_gb300.so).

Functions carry the C names and only marshal arguments: numpy arrays for host pointers,
torch tensors (or raw integer addresses) for device pointers, torch streams for cudaStream_t.
A negative status raises FdlbmError carrying the code and fdlbm_last_error(). Every step of
the method runs in the library's CUDA kernels; there is no other path. If the library cannot
be loaded the import of this module's functions fails loudly.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfdlbm_gb300.so")

FDLBM_OK, FDLBM_E_ARG, FDLBM_E_OOM, FDLBM_E_CUDA, FDLBM_E_NUMERIC, FDLBM_E_TIMEOUT, FDLBM_E_STATE, FDLBM_E_IO = \
    0, -1, -2, -3, -4, -5, -6, -7
FDLBM_BC_PERIODIC, FDLBM_BC_OUTFLOW, FDLBM_BC_DIRICHLET, FDLBM_BC_WALL, FDLBM_BC_HALO = 0, 1, 2, 3, 4
FDLBM_LEFT, FDLBM_RIGHT, FDLBM_BOTTOM, FDLBM_TOP = 0, 1, 2, 3
FDLBM_FP64, FDLBM_FP32_STORE, FDLBM_FNEQ32, FDLBM_FP32_STORE_DW, FDLBM_FP64_STRICT = 0, 1, 2, 3, 4
FDLBM_NO_LW, FDLBM_NO_DISP, FDLBM_NO_VISC, FDLBM_SWITCH_CONST = 1, 2, 4, 8
FDLBM_HEALTH_NUMERIC, FDLBM_HEALTH_KAPPA, FDLBM_HEALTH_TIMEOUT = 1, 2, 4
Q = 33


class FdlbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fdlbm error %d: %s" % (code, msg))
        self.code = code


class fdlbm_config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dt", ctypes.c_double), ("tau", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("bc", ctypes.c_int * 4), ("prec", ctypes.c_int), ("flags", ctypes.c_int)]


class fdlbm_request(ctypes.Structure):
    _fields_ = [("cfg", fdlbm_config), ("bstate", (ctypes.c_double * 4) * 4),
                ("rho", ctypes.POINTER(ctypes.c_double)), ("u", ctypes.POINTER(ctypes.c_double)),
                ("v", ctypes.POINTER(ctypes.c_double)), ("T", ctypes.POINTER(ctypes.c_double)),
                ("steps", ctypes.c_long), ("sim_fail_step", ctypes.c_long)]


class fdlbm_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("done", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("queued", ctypes.c_longlong), ("rounds", ctypes.c_longlong), ("max_active", ctypes.c_int),
                ("max_bytes", ctypes.c_size_t), ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double),
                ("mean_s", ctypes.c_double), ("wall_s", ctypes.c_double), ("aggregate_glups", ctypes.c_double)]


FDLBM_REQ_QUEUED, FDLBM_REQ_ACTIVE, FDLBM_REQ_DONE, FDLBM_REQ_FAILED, FDLBM_REQ_CANCELLED = 0, 1, 2, 3, 4
FDLBM_ENGINE_GPU, FDLBM_ENGINE_SIMULATED, FDLBM_ENGINE_GPU_SEPARATE = 0, 1, 2

_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def lib():
    """Load libfdlbm_gb300.so (building it first if sources changed and nvcc is present)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH) or os.environ.get("FDLBM_AUTOBUILD", "1") == "1":
            try:
                from . import build as _b
                _b.build()
            except RuntimeError:
                if not os.path.exists(LIB_PATH):
                    raise
        if not os.path.exists(LIB_PATH):
            raise ImportError("libfdlbm_gb300.so is missing; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        cfgp = ctypes.POINTER(fdlbm_config)
        sig = {
            "fdlbm_device_bytes": (ctypes.c_size_t, [cfgp]),
            "fdlbm_create_ex": (ctypes.c_int, [ctypes.POINTER(_VP), cfgp, _VP, ctypes.c_size_t, _VP]),
            "fdlbm_set_boundary_segment": (ctypes.c_int, [_VP, ctypes.c_int] + [ctypes.c_double] * 2 +
                                           [ctypes.c_int] + [ctypes.c_double] * 4),
            "fdlbm_clear_boundary_segment": (ctypes.c_int, [_VP, ctypes.c_int]),
            "fdlbm_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 +
                             [ctypes.POINTER(ctypes.c_int), ctypes.c_int, _VP]),
            "fdlbm_set_boundary_state": (ctypes.c_int, [_VP, ctypes.c_int] + [ctypes.c_double] * 4),
            "fdlbm_set_macro": (ctypes.c_int, [_VP, _DP, _DP, _DP, _DP]),
            "fdlbm_set_macro_device": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
            "fdlbm_step": (ctypes.c_int, [_VP, ctypes.c_long]),
            "fdlbm_sync": (ctypes.c_int, [_VP]),
            "fdlbm_get_macro": (ctypes.c_int, [_VP, _DP, _DP, _DP, _DP]),
            "fdlbm_get_macro_device": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
            "fdlbm_get_f": (ctypes.c_int, [_VP, _DP]),
            "fdlbm_set_f": (ctypes.c_int, [_VP, _DP]),
            "fdlbm_get_f_region": (ctypes.c_int, [_VP] + [ctypes.c_int] * 4 + [_DP]),
            "fdlbm_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
            "fdlbm_load": (ctypes.c_int, [_VP, ctypes.c_char_p]),
            "fdlbm_variant_count": (ctypes.c_int, []),
            "fdlbm_set_variant": (ctypes.c_int, [_VP, ctypes.c_int]),
            "fdlbm_get_variant": (ctypes.c_int, [_VP]),
            "fdlbm_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
            "fdlbm_steps_done": (ctypes.c_long, [_VP]),
            "fdlbm_current_buffer": (ctypes.c_int, [_VP]),
            "fdlbm_health": (ctypes.c_uint, [_VP]),
            "fdlbm_destroy": (ctypes.c_int, [_VP]),
            "fdlbm_last_error": (ctypes.c_char_p, [_VP]),
            "fdlbm_version": (ctypes.c_char_p, []),
            "fdlbm_step_noalloc": (ctypes.c_int, [cfgp, _VP, _VP, ctypes.c_long, ctypes.POINTER(ctypes.c_long), _VP]),
            "fdlbm_selftest_wait": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
            "fdlbm_fp64_rate": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _VP]),
            "fdlbm_selftest_grid_barrier": (ctypes.c_int, [ctypes.c_int] * 3 + [ctypes.POINTER(ctypes.c_int)]),
            "fdlbm_vn_spectrum": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP, _VP]),
            "fdlbm_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), _VP]),
            "fdlbm_batch_add": (ctypes.c_int, [_VP, _VP]),
            "fdlbm_batch_remove": (ctypes.c_int, [_VP, _VP]),
            "fdlbm_batch_size": (ctypes.c_int, [_VP]),
            "fdlbm_batch_step": (ctypes.c_int, [_VP, ctypes.c_long]),
            "fdlbm_batch_sync": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint)]),
            "fdlbm_batch_set_variant": (ctypes.c_int, [_VP, ctypes.c_int]),
            "fdlbm_batch_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]),
            "fdlbm_batch_destroy": (ctypes.c_int, [_VP]),
            "fdlbm_batch_last_error": (ctypes.c_char_p, [_VP]),
            "fdlbm_server_create": (ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_size_t, ctypes.c_int, ctypes.c_long,
                                                   ctypes.c_int, _VP]),
            "fdlbm_server_submit": (ctypes.c_int, [_VP, ctypes.POINTER(fdlbm_request),
                                                   ctypes.POINTER(ctypes.c_longlong)]),
            "fdlbm_server_poll": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)]),
            "fdlbm_server_wait": (ctypes.c_int, [_VP, ctypes.c_longlong, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
            "fdlbm_server_result": (ctypes.c_int, [_VP, ctypes.c_longlong, _DP, _DP, _DP, _DP, _DP]),
            "fdlbm_server_stats": (ctypes.c_int, [_VP, ctypes.POINTER(fdlbm_server_stats_t)]),
            "fdlbm_server_destroy": (ctypes.c_int, [_VP]),
            "fdlbm_server_last_error": (ctypes.c_char_p, [_VP]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(h, rc):
    if rc < 0:
        raise FdlbmError(rc, fdlbm_last_error(h))
    return rc


def _hp(a):
    return a.ctypes.data_as(_DP)


def _host(a, n):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _dptr(t):
    """Device address of a torch tensor (or an int address)."""
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device arrays must be contiguous CUDA tensors")
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_config(nx, ny, dx, dy, dt, tau, lam, bc, prec=FDLBM_FP64, flags=0):
    c = fdlbm_config()
    c.nx, c.ny, c.dx, c.dy, c.dt, c.tau, c.lambda_ = int(nx), int(ny), dx, dy, dt, tau, lam
    for i in range(4):
        c.bc[i] = int(bc[i])
    c.prec, c.flags = int(prec), int(flags)
    return c


def fdlbm_device_bytes(cfg):
    return int(lib().fdlbm_device_bytes(ctypes.byref(cfg)))


def fdlbm_create_ex(cfg, device_mem=None, device_bytes=0, stream=None):
    h = _VP()
    rc = lib().fdlbm_create_ex(ctypes.byref(h), ctypes.byref(cfg), None if device_mem is None else _dptr(device_mem),
                               int(device_bytes), _stream_ptr(stream))
    _check(None, rc)
    return h.value


def fdlbm_create(nx, ny, dx, dy, dt, tau, lam, bc, prec=FDLBM_FP64, stream=None):
    h = _VP()
    bc_arr = (ctypes.c_int * 4)(*[int(b) for b in bc])
    rc = lib().fdlbm_create(ctypes.byref(h), int(nx), int(ny), dx, dy, dt, tau, lam, bc_arr, int(prec),
                            _stream_ptr(stream))
    _check(None, rc)
    return h.value


def fdlbm_set_boundary_state(h, side, rho, u, v, T):
    return _check(h, lib().fdlbm_set_boundary_state(h, int(side), rho, u, v, T))


def fdlbm_set_boundary_segment(h, side, c0, speed, lower, rho, u, v, T):
    return _check(h, lib().fdlbm_set_boundary_segment(h, int(side), float(c0), float(speed), int(bool(lower)),
                                                       float(rho), float(u), float(v), float(T)))


def fdlbm_clear_boundary_segment(h, side):
    return _check(h, lib().fdlbm_clear_boundary_segment(h, int(side)))


def fdlbm_set_macro(h, rho, u, v, T, n=None):
    n = n if n is not None else np.asarray(rho).size
    arrs = [_host(a, n) for a in (rho, u, v, T)]
    return _check(h, lib().fdlbm_set_macro(h, *[_hp(a) for a in arrs]))


def fdlbm_set_macro_device(h, rho, u, v, T):
    return _check(h, lib().fdlbm_set_macro_device(h, *[_dptr(a) for a in (rho, u, v, T)]))


def fdlbm_step(h, nsteps):
    return _check(h, lib().fdlbm_step(h, int(nsteps)))


def fdlbm_sync(h):
    return _check(h, lib().fdlbm_sync(h))


def fdlbm_get_macro(h, nx, ny, check=True):
    out = [np.empty((ny, nx)) for _ in range(4)]
    rc = lib().fdlbm_get_macro(h, *[_hp(a) for a in out])
    if check:
        _check(h, rc)
    return tuple(out)


def fdlbm_get_macro_device(h, rho, u, v, T):
    return _check(h, lib().fdlbm_get_macro_device(h, *[_dptr(a) for a in (rho, u, v, T)]))


def fdlbm_get_f(h, nx, ny):
    f = np.empty((Q, ny, nx))
    _check(h, lib().fdlbm_get_f(h, _hp(f)))
    return f


def fdlbm_get_f_region(h, x0, y0, w, hgt):
    f = np.empty((Q, hgt, w))
    _check(h, lib().fdlbm_get_f_region(h, int(x0), int(y0), int(w), int(hgt), _hp(f)))
    return f


def fdlbm_set_f(h, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    return _check(h, lib().fdlbm_set_f(h, _hp(f)))


def fdlbm_save(h, path):
    return _check(h, lib().fdlbm_save(h, os.fsencode(path)))


def fdlbm_load(h, path):
    return _check(h, lib().fdlbm_load(h, os.fsencode(path)))


def fdlbm_variant_count():
    return int(lib().fdlbm_variant_count())


def fdlbm_set_variant(h, variant):
    return _check(h, lib().fdlbm_set_variant(h, int(variant)))


def fdlbm_get_variant(h):
    return _check(h, lib().fdlbm_get_variant(h))


def fdlbm_autotune(h, trial_steps=5):
    """Returns the per-variant mean launch times (ms); the handle keeps the fastest variant."""
    n = fdlbm_variant_count()
    times = (ctypes.c_float * n)()
    _check(h, lib().fdlbm_autotune(h, int(trial_steps), times))
    return list(times)


def fdlbm_current_buffer(h):
    return _check(h, lib().fdlbm_current_buffer(h))


def fdlbm_steps_done(h):
    return int(lib().fdlbm_steps_done(h))


def fdlbm_fp64_rate(iters=20000, stream=None):
    """Measured FP64 operations per second (fused multiply-add chains at full occupancy)."""
    r = ctypes.c_double(0.0)
    rc = lib().fdlbm_fp64_rate(int(iters), ctypes.byref(r), _stream_ptr(stream))
    if rc != FDLBM_OK:
        raise FdlbmError(rc, "fdlbm_fp64_rate failed")
    return r.value


def fdlbm_selftest_grid_barrier(skip, iters, rounds=4):
    """(status, completed) of the persistent variants' grid-barrier self-test."""
    done = ctypes.c_int(-1)
    rc = lib().fdlbm_selftest_grid_barrier(int(skip), int(iters), int(rounds), ctypes.byref(done))
    return rc, done.value


def fdlbm_selftest_wait(arrive, iters):
    """(status, completed) of the bounded mbarrier wait's self-test (no exception on a timeout:
    that is the expected outcome without an arrival)."""
    done = ctypes.c_int(-1)
    rc = lib().fdlbm_selftest_wait(int(arrive), int(iters), ctypes.byref(done))
    return rc, done.value


def fdlbm_health(h):
    return int(lib().fdlbm_health(h))


def fdlbm_destroy(h):
    return lib().fdlbm_destroy(h)


def fdlbm_last_error(h):
    s = lib().fdlbm_last_error(h)
    return s.decode() if s else ""


def _bcheck(b, rc):
    if rc < 0:
        raise FdlbmError(rc, fdlbm_batch_last_error(b))
    return rc


def fdlbm_batch_create(stream=None):
    b = _VP()
    _bcheck(None, lib().fdlbm_batch_create(ctypes.byref(b), _stream_ptr(stream)))
    return b.value


def fdlbm_batch_add(b, h):
    return _bcheck(b, lib().fdlbm_batch_add(b, h))


def fdlbm_batch_remove(b, h):
    return _bcheck(b, lib().fdlbm_batch_remove(b, h))


def fdlbm_batch_size(b):
    return _bcheck(b, lib().fdlbm_batch_size(b))


def fdlbm_batch_step(b, nsteps):
    return _bcheck(b, lib().fdlbm_batch_step(b, int(nsteps)))


def fdlbm_batch_sync(b):
    """Returns (number of members with a sticky error, per-member health words)."""
    n = max(1, fdlbm_batch_size(b))
    words = (ctypes.c_uint * n)()
    failed = _bcheck(b, lib().fdlbm_batch_sync(b, words))
    return failed, list(words)[:fdlbm_batch_size(b)]


def fdlbm_batch_set_variant(b, variant):
    return _bcheck(b, lib().fdlbm_batch_set_variant(b, int(variant)))


def fdlbm_batch_autotune(b, trial_steps=3):
    n = fdlbm_variant_count()
    times = (ctypes.c_float * n)()
    _bcheck(b, lib().fdlbm_batch_autotune(b, int(trial_steps), times))
    return list(times)


def fdlbm_batch_destroy(b):
    return lib().fdlbm_batch_destroy(b)


def fdlbm_batch_last_error(b):
    s = lib().fdlbm_batch_last_error(b)
    return s.decode() if s else ""


def _scheck(srv, rc):
    if rc < 0:
        raise FdlbmError(rc, fdlbm_server_last_error(srv))
    return rc


def fdlbm_server_create(budget_bytes, max_slots=256, round_steps=500, engine=FDLBM_ENGINE_GPU, stream=None):
    srv = _VP()
    _scheck(None, lib().fdlbm_server_create(ctypes.byref(srv), int(budget_bytes), int(max_slots), int(round_steps),
                                            int(engine), _stream_ptr(stream)))
    return srv.value


def fdlbm_server_submit(srv, cfg, rho, u, v, T, steps, bstate=None, sim_fail_step=0):
    n = cfg.nx * cfg.ny
    arrs = [_host(a, n) for a in (rho, u, v, T)]
    req = fdlbm_request()
    req.cfg = cfg
    if bstate is not None:
        for i in range(4):
            for j in range(4):
                req.bstate[i][j] = float(bstate[i][j])
    req.rho, req.u, req.v, req.T = [_hp(a) for a in arrs]
    req.steps = int(steps)
    req.sim_fail_step = int(sim_fail_step)
    rid = ctypes.c_longlong()
    _scheck(srv, lib().fdlbm_server_submit(srv, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def fdlbm_server_poll(srv, rid):
    st = ctypes.c_int()
    _scheck(srv, lib().fdlbm_server_poll(srv, int(rid), ctypes.byref(st)))
    return st.value


def fdlbm_server_wait(srv, rid, timeout_s=-1.0):
    """Returns the final status, or None if the timeout ran out first."""
    st = ctypes.c_int()
    rc = lib().fdlbm_server_wait(srv, int(rid), float(timeout_s), ctypes.byref(st))
    if rc == FDLBM_E_TIMEOUT:
        return None
    _scheck(srv, rc)
    return st.value


def fdlbm_server_result(srv, rid, nx, ny):
    """(rho, u, v, T, seconds_to_solution) of a finished request; raises FdlbmError for a failed one."""
    out = [np.empty((ny, nx)) for _ in range(4)]
    secs = ctypes.c_double()
    _scheck(srv, lib().fdlbm_server_result(srv, int(rid), *[_hp(a) for a in out], ctypes.byref(secs)))
    return tuple(out) + (secs.value,)


def fdlbm_server_stats(srv):
    st = fdlbm_server_stats_t()
    _scheck(srv, lib().fdlbm_server_stats(srv, ctypes.byref(st)))
    return {name: getattr(st, name) for name, _ in st._fields_}


def fdlbm_server_destroy(srv):
    return lib().fdlbm_server_destroy(srv)


def fdlbm_server_last_error(srv):
    s = lib().fdlbm_server_last_error(srv)
    return s.decode() if s else ""


FDLBM_NOALLOC_MAX_STEPS = 4096


def fdlbm_step_noalloc(cfg, f_a, f_b, nsteps, stream=None):
    """Allocation-free fused step on caller buffers; returns first_bad_step (-1 if none).

    Raises FdlbmError (FDLBM_E_NUMERIC carries the step in .first_bad_step)."""
    bad = ctypes.c_long(-1)
    rc = lib().fdlbm_step_noalloc(ctypes.byref(cfg), _dptr(f_a), _dptr(f_b), int(nsteps), ctypes.byref(bad),
                                  _stream_ptr(stream))
    if rc < 0:
        err = FdlbmError(rc, fdlbm_last_error(None))
        err.first_bad_step = bad.value
        raise err
    return bad.value


# ---- von Neumann analysis (Sec. 4, Eqs. 18-20)

FDLBM_VN_OK, FDLBM_VN_BAD_CASE, FDLBM_VN_NO_CONVERGENCE = 0, 1, 2

# numpy layout of struct fdlbm_vn_case (64 bytes)
VN_CASE = np.dtype([("rho", "f8"), ("ux", "f8"), ("uy", "f8"), ("T", "f8"), ("xi_x", "f8"), ("xi_y", "f8"),
                    ("lam", "f8"), ("flags", "i4"), ("reserved", "i4")])


def vn_cases(states, xi_x, xi_y, lam, flags=0):
    """Broadcast per-case arrays into a VN_CASE record array. states: (..., 4) rows (rho, u1, u2, T)."""
    st = np.asarray(states, dtype=np.float64)
    shape = np.broadcast_shapes(st.shape[:-1], np.shape(xi_x), np.shape(xi_y), np.shape(lam), np.shape(flags))
    out = np.zeros(int(np.prod(shape)), dtype=VN_CASE)
    st = np.broadcast_to(st, shape + (4,)).reshape(-1, 4)
    for k, name in enumerate(("rho", "ux", "uy", "T")):
        out[name] = st[:, k]
    out["xi_x"] = np.broadcast_to(xi_x, shape).ravel()
    out["xi_y"] = np.broadcast_to(xi_y, shape).ravel()
    out["lam"] = np.broadcast_to(lam, shape).ravel()
    out["flags"] = np.broadcast_to(flags, shape).ravel()
    return out


def fdlbm_vn_spectrum(cases, n, dx, dy, dt, tau, max_abs, omega=None, G=None, status=None, stream=None):
    """Raw call: every array argument is a CUDA tensor (or a device address)."""
    opt = [None if a is None else _dptr(a) for a in (omega, G, status)]
    rc = lib().fdlbm_vn_spectrum(_dptr(cases), int(n), float(dx), float(dy), float(dt), float(tau), _dptr(max_abs),
                                 *opt, _stream_ptr(stream))
    return _check(None, rc)


def vn_spectrum(cases, dx, dy, dt, tau, eigenvalues=False, matrix=False, device="cuda"):
    """Run fdlbm_vn_spectrum on a VN_CASE array and return host results:
    (max_abs (n,), status (n,), omega (n, 33) complex or None, G (n, 33, 33) complex or None)."""
    import torch
    cases = np.ascontiguousarray(cases, dtype=VN_CASE)
    n = cases.shape[0]
    d_cases = torch.from_numpy(cases.view(np.uint8).copy()).to(device)
    d_max = torch.empty(n, dtype=torch.float64, device=device)
    d_st = torch.empty(n, dtype=torch.int32, device=device)
    d_om = torch.empty(66 * n, dtype=torch.float64, device=device) if eigenvalues else None
    d_G = torch.empty(2178 * n, dtype=torch.float64, device=device) if matrix else None
    fdlbm_vn_spectrum(d_cases, n, dx, dy, dt, tau, d_max, d_om, d_G, d_st, torch.cuda.current_stream())
    om = d_om.cpu().numpy().view(np.complex128).reshape(n, 33) if eigenvalues else None
    G = d_G.cpu().numpy().view(np.complex128).reshape(n, 33, 33) if matrix else None
    return d_max.cpu().numpy(), d_st.cpu().numpy(), om, G


def fdlbm_version():
    return lib().fdlbm_version().decode()


class Solver:
    """One solve: owns a handle whose device memory is a torch uint8 tensor on the given stream."""

    def __init__(self, nx, ny, dx, dy, dt, tau, lam, bc, prec=FDLBM_FP64, flags=0, bstate=None, stream=None,
                 use_torch_memory=True):
        self.nx, self.ny = int(nx), int(ny)
        self.cfg = make_config(nx, ny, dx, dy, dt, tau, lam, bc, prec, flags)
        self._mem = None
        nbytes = fdlbm_device_bytes(self.cfg)
        if nbytes == 0:
            raise FdlbmError(FDLBM_E_ARG, "invalid configuration")
        if use_torch_memory:
            import torch
            self._mem = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self._mem.data_ptr()
            aligned = (base + 255) // 256 * 256
            self.mem_offset = aligned - base  # the handle's buffers start here in self._mem
            self.h = fdlbm_create_ex(self.cfg, aligned, nbytes, stream)
        else:
            self.h = fdlbm_create_ex(self.cfg, None, 0, stream)
        if bstate is not None:
            for side in range(4):
                if int(bc[side]) == FDLBM_BC_DIRICHLET:
                    fdlbm_set_boundary_state(self.h, side, *[float(x) for x in bstate[side]])

    @classmethod
    def from_workload(cls, w, prec=FDLBM_FP64, flags=0, stream=None, use_torch_memory=True):
        s = cls(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, prec, flags, w.bstate, stream, use_torch_memory)
        for side, c0, speed, lower, st in w.meta.get("segments", ()):
            fdlbm_set_boundary_segment(s.h, side, c0, speed, lower, *st)
        s.set_macro(*w.macros())
        return s

    def set_macro(self, rho, u, v, T):
        n = self.nx * self.ny
        return fdlbm_set_macro(self.h, rho, u, v, T, n)

    def step(self, n):
        return fdlbm_step(self.h, n)

    def sync(self):
        return fdlbm_sync(self.h)

    def get_macro(self, check=True):
        return fdlbm_get_macro(self.h, self.nx, self.ny, check)

    def get_f(self):
        return fdlbm_get_f(self.h, self.nx, self.ny)

    def set_f(self, f):
        return fdlbm_set_f(self.h, f)

    def get_f_region(self, x0, y0, w, hgt):
        return fdlbm_get_f_region(self.h, x0, y0, w, hgt)

    def set_variant(self, v):
        return fdlbm_set_variant(self.h, v)

    def autotune(self, trial_steps=5):
        return fdlbm_autotune(self.h, trial_steps)

    @property
    def steps_done(self):
        return fdlbm_steps_done(self.h)

    def health(self):
        return fdlbm_health(self.h)

    def close(self):
        if getattr(self, "h", None):
            fdlbm_destroy(self.h)
            self.h = None
        self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
