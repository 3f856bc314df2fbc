"""Slab decomposition of one grid over several ranks, with a 2-row ghost exchange per step.

A grid of nx x NY nodes is cut along y into one slab of rows per rank. A side where a slab borders
another slab takes the boundary kind HALO: the library never writes those ghost rows; after every
step each rank copies its two edge rows of the current state into the neighbour's ghost rows with
point-to-point send/receive (torch.distributed: NCCL between GPUs, gloo between CPU processes).
Eq. 17 reaches I +- 2, and the switch of Eq. 16 the moments at I +- 1, which a rank takes from the
ghost f, so two rows per side are the whole exchange: no collective, no moment exchange. Each
node's arithmetic is then that of the single grid, bit for bit.

The GPU path runs each rank's slab with the library's own step (SlabSolver); the exchange is a
function of plain tensors [planes, rows, width] so that it serves any state layout, a CPU
restatement included. One GPU per process; remote rows arrive in local buffers first (no
multicast).
"""
from . import fdlbm as F

NG = 2


def slab_rows(ny, world, rank):
    """[j0, j1): the rows of the global grid that rank owns (contiguous, sizes differing by <= 1)."""
    base, extra = divmod(ny, world)
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def neighbours(world, rank, periodic_y):
    """(below, above) ranks, None where the slab touches the grid's own bottom or top side."""
    below = rank - 1 if rank > 0 else (world - 1 if periodic_y else None)
    above = rank + 1 if rank < world - 1 else (0 if periodic_y else None)
    return below, above


def slab_bc(bc, world, rank):
    """The slab's boundary kinds: the grid's own on its outer sides, HALO where it meets a slab
    (with periodic y every side between slabs is HALO, including the wrap-around)."""
    periodic_y = bc[2] == F.FDLBM_BC_PERIODIC
    if world == 1:
        return tuple(bc)
    below, above = neighbours(world, rank, periodic_y)
    bottom = F.FDLBM_BC_HALO if below is not None else bc[2]
    top = F.FDLBM_BC_HALO if above is not None else bc[3]
    return (bc[0], bc[1], bottom, top)


def exchange_ghost_rows(planes, below, above, dist, group=None):
    """One ghost exchange on state tensors of shape [P, ny + 4, width] (ghost rows 0-1 and
    ny + 2 - ny + 3 around interior rows 2 .. ny + 1).

    Sends interior rows 2-3 to `below` (they become its top ghost rows) and rows ny - ny + 1 to
    `above` (its bottom ghost rows); receives the same from them. `below` / `above` are ranks or
    None. `planes` may be one tensor or a list of tensors with the same row layout (all of a state's
    parts, e.g. g and the macros of FDLBM_FNEQ32); the tensors are updated in place."""
    parts = planes if isinstance(planes, (list, tuple)) else [planes]
    # Sends first (bottom rows, then top rows, per part), then receives in the order that pairs
    # them when one neighbour is both below and above (two ranks, periodic y): NCCL matches
    # messages between two ranks by their order, gloo by their tags, and both orders agree.
    sends, recvs, recv = [], [], []
    for k, t in enumerate(parts):
        ny = t.shape[1] - 2 * NG
        if below is not None:
            sends.append(dist.P2POp(dist.isend, t[:, NG:2 * NG, :].contiguous(), below, group, tag=2 * k))
        if above is not None:
            sends.append(dist.P2POp(dist.isend, t[:, ny:ny + NG, :].contiguous(), above, group, tag=2 * k + 1))
    for k, t in enumerate(parts):
        ny = t.shape[1] - 2 * NG
        if above is not None:  # the rank above sent its bottom rows: my top ghost rows
            buf = torch_empty_like(t[:, 0:NG, :])
            recvs.append(dist.P2POp(dist.irecv, buf, above, group, tag=2 * k))
            recv.append((t, ny + NG, buf))
        if below is not None:  # the rank below sent its top rows: my bottom ghost rows
            buf = torch_empty_like(t[:, 0:NG, :])
            recvs.append(dist.P2POp(dist.irecv, buf, below, group, tag=2 * k + 1))
            recv.append((t, 0, buf))
    ops = sends + recvs
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for t, row, buf in recv:
        t[:, row:row + NG, :].copy_(buf)


def torch_empty_like(t):
    import torch
    return torch.empty_like(t)


class SlabSolver:
    """One rank's slab of a grid split along y, stepped by the library with a ghost exchange after
    every step. fields: the global (rho, u, v, T), ny x nx each (only the slab's rows are used).
    The slab's Solver runs on torch's current CUDA stream, so the exchange is ordered after it."""

    def __init__(self, nx, ny, dx, dy, dt, tau, lam, bc, fields, dist, prec=F.FDLBM_FP64, bstate=None):
        import torch
        self.dist = dist
        world, rank = dist.get_world_size(), dist.get_rank()
        self.j0, self.j1 = slab_rows(ny, world, rank)
        self.below, self.above = neighbours(world, rank, bc[2] == F.FDLBM_BC_PERIODIC)
        if world == 1:
            self.below = self.above = None
        self.bc = slab_bc(bc, world, rank)
        self.prec = prec
        self.solver = F.Solver(nx, self.j1 - self.j0, dx, dy, dt, tau, lam, self.bc, prec, 0, bstate,
                               stream=torch.cuda.current_stream())
        self.solver.set_macro(*[a[self.j0:self.j1] for a in fields])
        self._exchange()

    def _views(self):
        """The current state as tensors [P, rows, pitch] over the solver's torch memory."""
        import torch
        s = self.solver
        nx, ny = s.nx, s.ny
        pitch = (nx + 2 * NG + 31) // 32 * 32
        rows = ny + 2 * NG
        plane = pitch * rows
        esize = 8 if self.prec == F.FDLBM_FP64 else 4
        gbytes = (33 * plane * esize + 255) // 256 * 256
        fbytes = gbytes
        if self.prec == F.FDLBM_FNEQ32:
            fbytes = (gbytes + 4 * plane * 8 + 255) // 256 * 256
        base = s.mem_offset + F.fdlbm_current_buffer(s.h) * fbytes
        mem = s._mem
        dt = torch.float64 if self.prec == F.FDLBM_FP64 else torch.float32
        parts = [mem[base:base + 33 * plane * esize].view(dt).view(33, rows, pitch)]
        if self.prec == F.FDLBM_FNEQ32:
            parts.append(mem[base + gbytes:base + gbytes + 4 * plane * 8].view(torch.float64).view(4, rows, pitch))
        return parts

    def _exchange(self):
        if self.below is None and self.above is None:
            return
        exchange_ghost_rows(self._views(), self.below, self.above, self.dist)

    def step(self, n=1):
        for _ in range(int(n)):
            self.solver.step(1)
            self._exchange()

    def get_macro(self):
        return self.solver.get_macro()
