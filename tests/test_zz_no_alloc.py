"""fdlbm_step_noalloc: the fused step for callers that cannot allocate device memory.

Such a caller (its device memory all belongs to another allocator, or its path must not call
cudaMalloc) owns both state buffers; the entry point keeps its only scratch, one health word
per step, in a static device array. These tests check it against the handle path
(fdlbm_step) on two calls in a row, within the f-level tolerance the parity tests use, on grids
that take each kind of launch the entry point can pick (ring-parallel for small grids, the 32 x 8
tile, the 32 x 16 tile that stages f_eq in dynamic shared memory, a tile holding a periodic tube's
height), check that a call changes the device's free memory by nothing, and check its size limit
and its report of the failing step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    F.lib()


def _layout(cfg):
    pitch = (cfg.nx + 4 + 31) // 32 * 32
    rows = cfg.ny + 4
    esize = 8 if cfg.prec == F.FDLBM_FP64 else 4
    fbytes = (33 * pitch * rows * esize + 255) // 256 * 256
    if cfg.prec == F.FDLBM_FNEQ32:  # then 4 FP64 planes of the macros
        fbytes = (fbytes + 4 * pitch * rows * 8 + 255) // 256 * 256
    return pitch, rows, esize, fbytes


def _interior(buf, cfg):
    """The stored values of the interior: f, or for FNEQ32 its departure g (the tests compare the
    buffers, which the handle and the entry point fill the same way)."""
    pitch, rows, esize, _ = _layout(cfg)
    dt = torch.float64 if esize == 8 else torch.float32
    a = buf[:33 * pitch * rows * esize].view(dt).reshape(33, rows, pitch)
    out = a[:, 2:2 + cfg.ny, 2:2 + cfg.nx].double().cpu().numpy()
    if cfg.prec == F.FDLBM_FNEQ32:
        g0 = (33 * pitch * rows * 4 + 255) // 256 * 256
        m = buf[g0:g0 + 4 * pitch * rows * 8].view(torch.float64).reshape(4, rows, pitch)
        out = np.concatenate([out, m[:, 2:2 + cfg.ny, 2:2 + cfg.nx].cpu().numpy()])
    return out


def _handle_state(s):
    """The handle's current buffer, read the same way as the entry point's."""
    _, _, _, fbytes = _layout(s.cfg)
    torch.cuda.synchronize()
    off = s.mem_offset + F.fdlbm_current_buffer(s.h) * fbytes
    return _interior(s._mem[off:off + fbytes], s.cfg)


def _copies(solver):
    """Two caller-owned device buffers holding the handle's pair: the current state and the
    second buffer, whose interior the first step writes (both carry the Dirichlet ghosts)."""
    _, _, _, fbytes = _layout(solver.cfg)
    off = solver.mem_offset
    bufs = []
    for b in range(2):
        t = torch.empty(fbytes, dtype=torch.uint8, device="cuda")
        assert t.data_ptr() % 256 == 0
        t.copy_(solver._mem[off + b * fbytes: off + (b + 1) * fbytes])
        bufs.append(t)
    torch.cuda.synchronize()
    return bufs


# (workload, precision): the launch each grid takes is the library's default for its size
CASES = {
    "ring_parallel_4096_fp64": (lambda: W.riemann4q(n=64), F.FDLBM_FP64),          # <= 6144 sites
    "ring_parallel_4096_fp32": (lambda: W.riemann4q(n=64), F.FDLBM_FP32_STORE),
    "tile32x8_reflection_fp64": (lambda: W.reflection(nx=300, ny=75), F.FDLBM_FP64),  # 22 500 sites
    "tile32x8_riemann_fp32": (lambda: W.riemann4q(n=128), F.FDLBM_FP32_STORE),
    "tube_wrap_4000x4_fp64": (lambda: W.shock_tube(nx=4000, ny=4), F.FDLBM_FP64),     # 4-row tube
    "staged32x16_262144_fp32": (lambda: W.riemann4q(n=512), F.FDLBM_FP32_STORE),    # > 200 000 sites
    "tile32x16_262144_fp64": (lambda: W.riemann4q(n=512), F.FDLBM_FP64),
    "fneq32_reflection": (lambda: W.reflection(nx=300, ny=75), F.FDLBM_FNEQ32),
    "fp32dw_staged_262144": (lambda: W.riemann4q(n=512), F.FDLBM_FP32_STORE_DW),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_matches_handle_on_two_calls(case):
    make, prec = CASES[case]
    w = make()
    s = F.Solver.from_workload(w, prec)
    a, b = _copies(s)
    # call 1: 7 steps, result in the second buffer (odd count)
    s.step(7)
    ref = _handle_state(s)
    assert F.fdlbm_step_noalloc(s.cfg, a, b, 7) == -1
    torch.cuda.synchronize()
    got = _interior(b, s.cfg)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
    # call 2: 4 more steps from that result, even count -> result stays in the first argument
    s.step(4)
    ref = _handle_state(s)
    assert F.fdlbm_step_noalloc(s.cfg, b, a, 4) == -1
    torch.cuda.synchronize()
    got = _interior(b, s.cfg)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.abs(ref).max()
    s.close()


@pytest.mark.parametrize("prec", [F.FDLBM_FP64, F.FDLBM_FP32_STORE])
def test_noalloc_call_leaves_free_device_memory_unchanged(prec):
    """After a first call (which may load the module and look up the scratch address), a call
    on a grid that takes the staged 32 x 16 tile changes the device's free memory by 0 bytes."""
    w = W.riemann4q(n=512)
    s = F.Solver.from_workload(w, prec)
    a, b = _copies(s)
    assert F.fdlbm_step_noalloc(s.cfg, a, b, 2) == -1
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert F.fdlbm_step_noalloc(s.cfg, a, b, 3) == -1
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    s.close()


def test_noalloc_rejects_too_many_steps():
    w = W.sod(nx=64, ny=4)
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    a, b = _copies(s)
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_step_noalloc(s.cfg, a, b, F.FDLBM_NOALLOC_MAX_STEPS + 1)
    assert ei.value.code == F.FDLBM_E_ARG
    assert "FDLBM_NOALLOC_MAX_STEPS" in F.fdlbm_last_error(None)


def test_noalloc_reports_the_failing_step():
    """Shock Mach 20 into gas at rest: the input of step 1 (after one step) holds T <= 0."""
    w = W.shock_tube(nx=200, ny=4, steps=3, Ms=20.0, U=0.0, T1=1.0, lam=5.0)
    s = F.Solver.from_workload(w, F.FDLBM_FP64)
    a, b = _copies(s)
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_step_noalloc(s.cfg, a, b, 3)
    assert ei.value.code == F.FDLBM_E_NUMERIC
    assert ei.value.first_bad_step == 1
