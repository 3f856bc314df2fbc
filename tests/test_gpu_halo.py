"""The slab solver's GPU path (paper_0801_4169_gb300/halo.py SlabSolver) on one GPU.

Every run here gets one GPU, so two slabs are two solves in one process, each driven by its own
thread. Their exchange goes through an in-process stand-in for torch.distributed's point-to-point
calls (a mailbox keyed by source, destination and tag). No kernel waits on another, and the
library's launches of both slabs are ordered on the device. The slabs' interiors must equal the
single-grid GPU solve bit for bit, in every precision. This checks the slab solver's views of the
library's buffers (layout, current buffer, FNEQ32's two parts), not NCCL.
"""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_0801_4169_gb300 import fdlbm as F  # noqa: E402
from paper_0801_4169_gb300 import halo  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    F.lib()


class _Mailbox:
    def __init__(self):
        self.cv = threading.Condition()
        self.box = {}


class _LocalDist:
    """Enough of torch.distributed's point-to-point interface for halo.exchange_ghost_rows."""

    class P2POp:
        def __init__(self, op, tensor, peer, group=None, tag=0):
            self.op, self.tensor, self.peer, self.tag = op, tensor, peer, tag

    isend, irecv = "isend", "irecv"

    def __init__(self, mailbox, rank, world):
        self.mb, self.rank, self.world = mailbox, rank, world

    def get_rank(self):
        return self.rank

    def get_world_size(self):
        return self.world

    def batch_isend_irecv(self, ops):
        torch.cuda.synchronize()
        with self.mb.cv:
            for o in ops:
                if o.op == self.isend:
                    self.mb.box.setdefault((self.rank, o.peer, o.tag), []).append(o.tensor.clone())
            self.mb.cv.notify_all()
        mine = self

        class _Req:
            def wait(self_inner):
                with mine.mb.cv:
                    for o in ops:
                        if o.op != mine.irecv:
                            continue
                        key = (o.peer, mine.rank, o.tag)
                        ok = mine.mb.cv.wait_for(lambda: mine.mb.box.get(key), timeout=60)
                        assert ok, "no message %s" % (key,)
                        o.tensor.copy_(mine.mb.box[key].pop(0))
                torch.cuda.synchronize()

        return [_Req()]


def _fields(nx, ny):
    rng = np.random.default_rng(5)
    x = 2 * np.pi * (np.arange(nx) + 0.5) / nx
    y = 2 * np.pi * (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    out = []
    for b in (1.0, 0.3, -0.2, 1.0):
        a1, a2, p1, p2 = rng.uniform(-1, 1, 4)
        out.append(b + 0.15 * (abs(b) + 0.5) * (a1 * np.sin(X + p1) + a2 * np.cos(2 * Y + X + p2)))
    return out


@pytest.mark.parametrize("prec", [F.FDLBM_FP64, F.FDLBM_FP32_STORE, F.FDLBM_FNEQ32])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 3, 1)])
def test_two_slabs_equal_the_single_grid(prec, bc):
    nx, ny, steps = 70, 52, 15
    args = (1e-3, 1e-3, 1e-5, 1.5e-5, 1.5)
    fields = _fields(nx, ny)
    ref = F.Solver(nx, ny, *args, bc, prec)
    ref.set_macro(*fields)
    ref.step(steps)
    want = ref.get_f()
    mb = _Mailbox()
    out, err = {}, []

    def rank_main(rank):
        try:
            torch.cuda.set_device(0)
            sl = halo.SlabSolver(nx, ny, *args, bc, fields, _LocalDist(mb, rank, 2), prec=prec)
            sl.step(steps)
            out[rank] = (sl.j0, sl.j1, sl.solver.get_f())
        except Exception as e:  # reported below
            err.append(repr(e))

    th = [threading.Thread(target=rank_main, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=120)
    assert not err, err
    for rank in range(2):
        j0, j1, f = out[rank]
        assert np.array_equal(f, want[:, j0:j1, :]), rank
