"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports every function
include/fdlbm.h declares, and rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0801_4169_gb300 import fdlbm as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            src = open(os.path.join(ROOT, "include", hdr)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fdlbm_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_function():
    L = F.lib()
    names = _declared()
    assert len(names) >= 19
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    missing = [n for n in sorted(_declared()) if not hasattr(F, n)]
    assert not missing, missing


def test_version_and_null_handle():
    assert "sm_103a" in F.fdlbm_version()
    assert F.fdlbm_destroy(None) == 0
    assert isinstance(F.fdlbm_last_error(None), str)
    assert F.fdlbm_steps_done(None) == -1


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=0), "nx and ny"),
    (dict(dt=0.0), "dx, dy, dt, tau"),
    (dict(lam=-1.0), "lambda"),
    (dict(prec=7), "prec"),
    (dict(bc=(0, 1, 0, 0)), "periodic x"),
    (dict(bc=(3, 3, 0, 0), nx=1), "wall in x"),
    (dict(bc=(1, 1, 3, 3), ny=1), "wall in y"),
])
def test_invalid_configs_are_rejected_without_a_device(kw, msg):
    args = dict(nx=8, ny=4, dx=1e-3, dy=1e-3, dt=1e-5, tau=1e-5, lam=1.0, bc=(1, 1, 0, 0), prec=0)
    args.update(kw)
    cfg = F.make_config(args["nx"], args["ny"], args["dx"], args["dy"], args["dt"], args["tau"], args["lam"],
                        args["bc"], args["prec"])
    assert F.fdlbm_device_bytes(cfg) == 0
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_create_ex(cfg)
    assert ei.value.code == F.FDLBM_E_ARG
    assert msg in F.fdlbm_last_error(None)


def test_device_bytes_layout():
    """Two padded f buffers (rows of 32-element pitch), a health word and macro staging."""
    cfg = F.make_config(400, 4, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, (1, 1, 0, 0), F.FDLBM_FP64)
    pitch = 416  # round_up(400 + 4, 32)
    fbytes = 33 * pitch * 8 * 8
    fbytes = (fbytes + 255) // 256 * 256
    stage = (4 * 400 * 4 * 8 + 255) // 256 * 256
    assert F.fdlbm_device_bytes(cfg) == 2 * fbytes + 256 + stage
    cfg32 = F.make_config(400, 4, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, (1, 1, 0, 0), F.FDLBM_FP32_STORE)
    assert F.fdlbm_device_bytes(cfg32) < F.fdlbm_device_bytes(cfg)


def test_null_pointers_rejected():
    with pytest.raises(F.FdlbmError) as ei:
        F._check(None, F.lib().fdlbm_step(None, 1))
    assert ei.value.code == F.FDLBM_E_ARG


def test_vn_case_layout_and_argument_checks_without_a_device():
    assert F.VN_CASE.itemsize == 64  # struct fdlbm_vn_case: 7 doubles + 2 ints
    assert F.fdlbm_vn_spectrum(0, 0, 1e-3, 1e-3, 1e-5, 1e-5, 0) == 0  # n = 0: nothing to do
    for bad in (dict(n=-1), dict(dt=0.0), dict(tau=float("nan")), dict(dx=-1.0)):
        a = dict(n=4, dx=1e-3, dy=1e-3, dt=1e-5, tau=1e-5)
        a.update(bad)
        with pytest.raises(F.FdlbmError) as ei:
            F.fdlbm_vn_spectrum(0, a["n"], a["dx"], a["dy"], a["dt"], a["tau"], 0)
        assert ei.value.code == F.FDLBM_E_ARG
    with pytest.raises(F.FdlbmError) as ei:  # NULL cases / max_abs
        F.fdlbm_vn_spectrum(0, 4, 1e-3, 1e-3, 1e-5, 1e-5, 0)
    assert ei.value.code == F.FDLBM_E_ARG and "required" in F.fdlbm_last_error(None)


def test_vn_cases_broadcast():
    c = F.vn_cases([(1.0, 2.0, 0.0, 1.0), (2.0, 30.0, 0.0, 1.0)], np.linspace(0.1, 1.0, 5)[:, None], 0.0, 0.5)
    assert c.shape == (10,) and np.all(c["reserved"] == 0) and c["ux"][1] == 30.0 and c["xi_x"][2] == c["xi_x"][3]
