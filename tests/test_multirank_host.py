"""The N > 1 path of bench.py on CPU: replicas aggregated over a world-size-2 gloo group (no GPU).

Every rank runs an independent replica; the job time is the slowest rank's and the work the sum,
so value = sum(work) / max(time) (weak scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank          # rank 1 is the slow one
    lups_local = 1e9 * (rank + 1)
    ms, work, glups = bench.aggregate_over_ranks(ms_local, lups_local, tdist)
    q.put((rank, ms, work, glups))
    tdist.destroy_process_group()


def test_replicas_aggregate_max_time_and_total_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, work, glups in out:
        assert ms == 15.0 and work == 3e9
        assert glups == pytest.approx(3e9 / 15e-3 / 1e9)
