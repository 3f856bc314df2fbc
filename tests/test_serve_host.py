"""Scheduling policy of the native serving runtime (fdlbm_server_*), run on CPU with the
simulated engine (no device work). The simulated engine fills a result with the number of steps
the solve took, and fails a solve on reaching its sim_fail_step."""
import threading
import time

import numpy as np
import pytest

from paper_0801_4169_gb300 import fdlbm as F
from paper_0801_4169_gb300 import serve
from paper_0801_4169_gb300 import workloads as W


def _w(nx=256, ny=4):
    return W.shock_tube(nx=nx, ny=ny, steps=1, Ms=3.0, U=1.0)


def _bytes(nx, ny=4):
    w = _w(nx, ny)
    return F.fdlbm_device_bytes(F.make_config(w.nx, w.ny, w.dx, w.dy, w.dt, w.tau, w.lam, w.bc, 0))


def test_every_request_finishes_with_its_own_step_count():
    srv = serve.Server(budget_bytes=1 << 30, round_steps=37, engine="sim")
    rng = np.random.default_rng(0)
    ids = {}
    for k in range(30):
        steps = int(rng.integers(1, 400))
        ids[srv.submit(_w(int(rng.integers(64, 512))), steps, 0)] = steps
    for rid, steps in ids.items():
        assert srv.wait(rid, 30.0) == F.FDLBM_REQ_DONE
        status, macros, secs, err = srv.result(rid)
        assert status == F.FDLBM_REQ_DONE and np.all(macros[0] == steps) and secs > 0
    st = srv.stats()
    assert st["done"] == 30 and st["failed"] == 0 and st["p99_s"] >= st["p50_s"] > 0
    srv.close()


def test_budget_and_slots_bound_admission():
    budget = 3 * _bytes(512)
    srv = serve.Server(budget_bytes=budget, max_slots=2, round_steps=50, engine="sim")
    ids = [srv.submit(_w(512), 200, 0) for _ in range(8)]
    for rid in ids:
        srv.wait(rid, 30.0)
    st = srv.stats()
    assert st["max_bytes"] <= budget and st["max_active"] <= 2 and st["done"] == 8
    srv.close()


def test_admission_follows_submission_order():
    """One slot: requests finish in the order they were submitted (each waits for the previous)."""
    srv = serve.Server(budget_bytes=1 << 30, max_slots=1, round_steps=1000, engine="sim")
    ids = [srv.submit(_w(1024), 2000, 0) for _ in range(5)]
    lat = []
    for rid in ids:
        srv.wait(rid, 30.0)
        lat.append(srv.result(rid)[2])
    assert all(b > a for a, b in zip(lat, lat[1:]))  # time to solution includes the queueing
    srv.close()


def test_failed_request_does_not_stop_the_others():
    srv = serve.Server(budget_bytes=1 << 30, round_steps=25, engine="sim")
    good = [srv.submit(_w(), 300, 0) for _ in range(4)]
    bad = srv.submit(_w(), 300, 0, sim_fail_step=120)
    for rid in good + [bad]:
        srv.wait(rid, 30.0)
    assert srv.poll(bad) == F.FDLBM_REQ_FAILED
    status, macros, secs, err = srv.result(bad)
    assert status == F.FDLBM_REQ_FAILED and "numerical" in err
    for rid in good:
        status, macros, secs, err = srv.result(rid)
        assert status == F.FDLBM_REQ_DONE and np.all(macros[0] == 300)
    assert srv.stats()["failed"] == 1
    srv.close()


def test_oversized_request_is_refused_at_once():
    srv = serve.Server(budget_bytes=_bytes(256) - 1, round_steps=25, engine="sim")
    rid = srv.submit(_w(256), 10, 0)
    assert srv.poll(rid) == F.FDLBM_REQ_FAILED
    with pytest.raises(F.FdlbmError) as ei:
        F.fdlbm_server_result(srv.h, rid, 256, 4)
    assert ei.value.code == F.FDLBM_E_OOM
    srv.close()


def test_concurrent_submitters():
    srv = serve.Server(budget_bytes=1 << 30, round_steps=40, engine="sim")
    ids, lock = [], threading.Lock()

    def client(k):
        for j in range(10):
            rid = srv.submit(_w(128 + k), 50 + j, 0)
            with lock:
                ids.append((rid, 50 + j))

    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert len({rid for rid, _ in ids}) == 40
    for rid, steps in ids:
        srv.wait(rid, 30.0)
        assert np.all(srv.result(rid)[1][0] == steps)
    srv.close()


def test_wait_times_out_and_destroy_cancels():
    srv = serve.Server(budget_bytes=1 << 30, max_slots=1, round_steps=100000, engine="sim")
    long_id = srv.submit(_w(4096, 64), 3000, 0)      # ~0.8 s of simulated work
    queued = srv.submit(_w(256), 10, 0)
    assert srv.wait(queued, 0.05) is None
    assert srv.poll(queued) == F.FDLBM_REQ_QUEUED
    srv.close()  # stops after the running round; the queued request is cancelled
    assert long_id != queued
