"""The slab decomposition's ghost exchange (paper_0801_4169_gb300/halo.py) on CPU ranks.

Two and three gloo processes split a grid along y; each advances its slab with the FP64 oracle,
whose HALO sides it leaves to the exchange, and calls the library's exchange_ghost_rows after every
step. Every value of the interior and of the slab's ghost rows must equal the single-grid oracle
bit for bit: each node's arithmetic sees exactly the inputs it sees on one grid. (The GPU path is
the same exchange around the library's step; it is unmeasured on hardware, since every run here
gets one GPU.)
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_0801_4169_gb300 import halo  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    x = 2 * np.pi * (np.arange(nx) + 0.5) / nx
    y = 2 * np.pi * (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for b in (1.0, 0.3, -0.2, 1.0):
        a1, a2, p1, p2 = rng.uniform(-1, 1, 4)
        out.append(b + 0.15 * (abs(b) + 0.5) * (a1 * np.sin(X + p1) + a2 * np.cos(2 * Y + X + p2)))
    return out


CASES = {
    "periodic": (64, 64, (0, 0, 0, 0), 20),
    "outflow_wall": (48, 45, (1, 1, 3, 1), 20),
}


def _worker(rank, world, port, case, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import fdlbm as O
        nx, ny, bc, steps = CASES[case]
        fields = _fields(nx, ny, 3)
        j0, j1 = halo.slab_rows(ny, world, rank)
        below, above = halo.neighbours(world, rank, bc[2] == 0)
        sbc = halo.slab_bc(bc, world, rank)
        s = O.Sim(nx, j1 - j0, 1e-3, 1e-3, 1e-5, 1.5e-5, 1.5, sbc)
        s.set_macro(*[a[j0:j1] for a in fields])

        def exchange():
            t = torch.from_numpy(s.get_f_padded())
            halo.exchange_ghost_rows(t, below, above, tdist)
            s.set_f_padded(t.numpy())

        exchange()
        for _ in range(steps):
            assert s.step(1) == 0
            exchange()
        q.put((rank, j0, j1, s.get_f_padded()))
    finally:
        tdist.destroy_process_group()


def _run(world, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_slab_rows_cover_the_grid():
    for ny in (1, 7, 64, 45):
        for world in (1, 2, 3, 5):
            if world > ny:
                continue
            rows = [halo.slab_rows(ny, world, r) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
            assert max(b - a for a, b in rows) - min(b - a for a, b in rows) <= 1
    assert halo.neighbours(3, 0, True) == (2, 1) and halo.neighbours(3, 0, False) == (None, 1)
    assert halo.slab_bc((1, 1, 3, 1), 2, 0) == (1, 1, 3, 4) and halo.slab_bc((1, 1, 3, 1), 2, 1) == (1, 1, 4, 1)


@pytest.mark.parametrize("world,case", [(2, "periodic"), (3, "periodic"), (2, "outflow_wall"), (3, "outflow_wall")])
def test_slabs_equal_the_single_grid_bit_for_bit(world, case):
    from oracle import fdlbm as O
    nx, ny, bc, steps = CASES[case]
    ref = O.Sim(nx, ny, 1e-3, 1e-3, 1e-5, 1.5e-5, 1.5, bc)
    ref.set_macro(*_fields(nx, ny, 3))
    assert ref.step(steps) == 0
    fp = ref.get_f_padded()
    for rank, j0, j1, got in _run(world, case):
        # interior rows and the two ghost rows on each side, interior columns
        want = fp[:, j0:j1 + 4, 2:2 + nx]
        assert np.array_equal(got[:, :, 2:2 + nx], want), (rank, j0, j1)
