"""Batched stepping and continuous-batching serving on the GPU.

A member of a batch must give bit for bit the result it gives alone:
- with different grids and boundary kinds;
- across odd step counts and graph-chunk boundaries;
- when members join and leave mid-run;
- when another member fails.
The serving loop's results must equal alone runs too.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import serve  # noqa: E402
from paper_0801_4169_gb300 import workloads as W  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    F.lib()


def _members(prec):
    """Solves of different sizes and boundary kinds that share the scheme constants."""
    out = []
    for k, (nx, ny, bc) in enumerate([(300, 4, (1, 1, 0, 0)), (1000, 4, (1, 1, 0, 0)), (77, 33, (0, 0, 3, 2)),
                                      (130, 61, (2, 1, 3, 1))]):
        w = W.shock_tube(nx=nx, ny=ny, Ms=3.0 + k, U=1.0 + k) if ny == 4 else W.riemann4q(n=nx, ny=ny, seed=k)
        w = W.Workload(w.name, nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, bc, 0, w.rho, w.u, w.v, w.T,
                       bstate=np.array([[1.0, 0.5, 0.0, 0.8]] * 4))
        out.append(w)
    return out


def _solver(w, prec):
    return F.Solver.from_workload(w, prec)


@pytest.mark.parametrize("prec", [F.FDLBM_FP64, F.FDLBM_FP32_STORE, F.FDLBM_FNEQ32])
def test_member_equals_alone_bitwise(prec):
    ws = _members(prec)
    alone = [_solver(w, prec) for w in ws]
    for s in alone:
        s.step(37)
    ref = [s.get_f() for s in alone]
    b = F.fdlbm_batch_create()
    inb = [_solver(w, prec) for w in ws]
    for s in inb:
        F.fdlbm_batch_add(b, s.h)
    F.fdlbm_batch_step(b, 37)  # 1 + 2 graph chunks of 16 + 4 plain launches ... parity crosses chunks
    failed, words = F.fdlbm_batch_sync(b)
    assert failed == 0 and len(words) == len(ws)
    for s, r in zip(inb, ref):
        assert s.steps_done == 37
        assert np.array_equal(s.get_f(), r)
    F.fdlbm_batch_destroy(b)


def test_membership_changes_midway():
    prec = F.FDLBM_FP64
    ws = _members(prec)
    b = F.fdlbm_batch_create()
    s0, s1, s2 = _solver(ws[0], prec), _solver(ws[1], prec), _solver(ws[2], prec)
    F.fdlbm_batch_add(b, s0.h)
    F.fdlbm_batch_step(b, 5)             # batch counter odd
    s1.step(3)                           # s1 joins with its own history (odd)
    F.fdlbm_batch_add(b, s1.h)
    F.fdlbm_batch_step(b, 20)
    F.fdlbm_batch_remove(b, s0.h)        # s0 leaves and continues alone
    s0.step(4)
    F.fdlbm_batch_add(b, s2.h)
    F.fdlbm_batch_step(b, 17)
    F.fdlbm_batch_sync(b)
    totals = {0: 29, 1: 40, 2: 17}
    for k, s in ((0, s0), (1, s1), (2, s2)):
        a = _solver(ws[k], prec)
        a.step(totals[k])
        assert s.steps_done == totals[k]
        assert np.array_equal(s.get_f(), a.get_f()), k
    F.fdlbm_batch_destroy(b)


def test_failed_member_is_isolated():
    prec = F.FDLBM_FP64
    ws = _members(prec)
    bad = W.shock_tube(nx=200, ny=4, Ms=20.0, U=0.0, T1=1.0, lam=2.0)
    bad = W.Workload(bad.name, 200, 4, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, bad.bc, 0, bad.rho, bad.u, bad.v, bad.T)
    b = F.fdlbm_batch_create()
    good = [_solver(ws[0], prec), _solver(ws[2], prec)]
    sb = _solver(bad, prec)
    for s in (good[0], sb, good[1]):
        F.fdlbm_batch_add(b, s.h)
    F.fdlbm_batch_step(b, 10)
    failed, words = F.fdlbm_batch_sync(b)
    assert failed == 1 and words[1] & F.FDLBM_HEALTH_NUMERIC and not (words[0] | words[2]) & F.FDLBM_HEALTH_NUMERIC
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_batch_step(b, 1)
    assert ei.value.code == F.FDLBM_E_STATE
    F.fdlbm_batch_remove(b, sb.h)
    with pytest.raises(F.FdlbmError) as ei:
        sb.sync()
    assert ei.value.code == F.FDLBM_E_NUMERIC
    F.fdlbm_batch_step(b, 6)
    F.fdlbm_batch_sync(b)
    for s, w in zip(good, (ws[0], ws[2])):
        a = _solver(w, prec)
        a.step(16)
        assert np.array_equal(s.get_f(), a.get_f())
    F.fdlbm_batch_destroy(b)


def test_guards():
    ws = _members(F.FDLBM_FP64)
    b = F.fdlbm_batch_create()
    s = _solver(ws[0], F.FDLBM_FP64)
    F.fdlbm_batch_add(b, s.h)
    other = _solver(ws[1], F.FDLBM_FP32_STORE)
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_batch_add(b, other.h)
    assert ei.value.code == F.FDLBM_E_ARG
    with pytest.raises(F.FdlbmError) as ei:
        s.step(1)
    assert ei.value.code == F.FDLBM_E_STATE
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_batch_add(b, s.h)
    assert ei.value.code == F.FDLBM_E_STATE
    s.close()  # destroy removes it from the batch
    assert F.fdlbm_batch_size(b) == 0
    F.fdlbm_batch_destroy(b)


def test_batch_autotune_keeps_state():
    ws = _members(F.FDLBM_FP32_STORE)
    b = F.fdlbm_batch_create()
    ss = [_solver(w, F.FDLBM_FP32_STORE) for w in ws]
    for s in ss:
        F.fdlbm_batch_add(b, s.h)
    F.fdlbm_batch_step(b, 3)
    F.fdlbm_batch_sync(b)
    before = [s.get_f() for s in ss]
    times = F.fdlbm_batch_autotune(b, 2)
    # the tile variants (0-7) are timed; the ring-parallel ones are single-solve only (reported 0)
    assert len(times) == F.fdlbm_variant_count() and all(t > 0 for t in times[:8])
    F.fdlbm_batch_sync(b)
    for s, f in zip(ss, before):
        assert np.array_equal(s.get_f(), f) and s.steps_done == 3
    F.fdlbm_batch_step(b, 5)
    F.fdlbm_batch_sync(b)
    for s, w in zip(ss, ws):
        a = _solver(w, F.FDLBM_FP32_STORE)
        a.step(8)
        assert np.array_equal(s.get_f(), a.get_f())
    F.fdlbm_batch_destroy(b)


def test_serving_results_equal_alone_runs():
    """Continuous batching in the native runtime: 24 requests arriving over time, mixed sizes, Mach
    numbers and precisions. Every finished request's moments equal those of the same solve run
    alone, for the batched engine and for the separate-launch baseline alike, and the two engines
    fail the same requests (FP32 storage on ill-conditioned states)."""
    reqs = W.serving_requests(n=24, seed=11, nx_range=(256, 2048), steps_range=(50, 400), mean_gap_s=0.002)
    outcomes = {}
    for engine in ("gpu", "separate"):
        srv = serve.Server(budget_bytes=64 << 20, round_steps=37, engine=engine)
        out, st = serve.replay(srv, [W.Request(**vars(r)) for r in reqs])
        srv.close()
        assert st["done"] + st["failed"] == len(reqs) and st["max_bytes"] <= 64 << 20
        outcomes[engine] = {r.rid: (status, macros) for (r, status, macros, secs, err) in out.values()}
    for r in reqs:
        sb, mb = outcomes["gpu"][r.rid]
        ss, ms = outcomes["separate"][r.rid]
        assert sb == ss
        if sb != F.FDLBM_REQ_DONE:
            assert r.prec == F.FDLBM_FP32_STORE  # only FP32 storage fails on these states
            continue
        a = F.Solver.from_workload(W.request_workload(r), r.prec)
        a.step(r.steps)
        ref = a.get_macro(check=False)
        for got_b, got_s, want in zip(mb, ms, ref):
            assert np.array_equal(got_b, want) and np.array_equal(got_s, want)


@pytest.mark.parametrize("prec", [F.FDLBM_FP64, F.FDLBM_FP32_STORE])
def test_periodic_y_members_with_rows_that_differ(prec):
    """Batched tiles that hold a y-periodic grid's whole height take the ghost rows' moments from
    the interior rows they copy. Members whose rows all differ (four-quadrant states, ny = 3..16,
    periodic in y) must still match their alone runs bit for bit in every tile variant."""
    ws = []
    for k, (nx, ny) in enumerate([(90, 4), (70, 3), (64, 8), (40, 16), (50, 5)]):
        w = W.riemann4q(n=nx, ny=ny, seed=10 + k)
        ws.append(W.Workload(w.name, nx, ny, 1e-3, 1e-3, 1e-5, 1e-5, 2.0, (1, 1, 0, 0), 0, w.rho, w.u, w.v, w.T))
    assert all(not np.array_equal(w.rho[0], w.rho[w.ny // 2]) for w in ws)
    ref = []
    for w in ws:
        a = _solver(w, prec)
        a.step(12)
        ref.append(a.get_f())
        a.close()
    for v in range(8):
        b = F.fdlbm_batch_create()
        inb = [_solver(w, prec) for w in ws]
        for s in inb:
            F.fdlbm_batch_add(b, s.h)
        F.fdlbm_batch_set_variant(b, v)
        F.fdlbm_batch_step(b, 12)
        failed, _ = F.fdlbm_batch_sync(b)
        assert failed == 0
        for s, r in zip(inb, ref):
            assert np.array_equal(s.get_f(), r), v
        F.fdlbm_batch_destroy(b)
        for s in inb:
            s.close()
