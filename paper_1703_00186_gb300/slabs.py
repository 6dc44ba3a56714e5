"""x-slab decomposition of one lattice over ranks (Sect. 4, Fig. "schedulingop").

The paper splits the 2-D lattice along x over N devices connected in a ring;
each rank holds a sub-lattice of about L_x / N columns surrounded by three
halo columns on each side.  At the start of every time step the pbc step
refills the halos with the three adjoining physical columns of the two ring
neighbours (37 populations, 3 columns each way), and the sites that read no
halo column (the bulk) are processed while that exchange is in flight; the
three leftmost and rightmost physical columns follow once it has completed.

Here a slab of w physical columns is a lattice of w + 6 columns (halo columns
0..2 and w+3..w+5, physical columns 3..w+2), stepped piecewise with
lbm_step_columns.  The halos travel through contiguous buffers
(lbm_pack_columns / lbm_unpack_columns) as point-to-point messages of
torch.distributed: NCCL between GPUs, gloo between CPU processes.  The ranks
exchange nothing else: there is no collective on the data path.

The exchange and the schedule are written against a small backend interface
(``LatticeBackend`` below for the GPU), so that the same protocol also runs
with CPU tensors.
"""
from __future__ import annotations

import torch

HX = 3  # halo columns on each side: the longest hop of the D2Q37 velocities


def partition(lx: int, world: int):
    """(x0, w) of every rank: contiguous column ranges covering 0..lx-1, the
    first lx % world ranks one column wider.  Every slab needs w >= 3 so that
    its halos come from its two ring neighbours only."""
    if world < 1 or lx < HX * world:
        raise ValueError(f"cannot split {lx} columns over {world} ranks with >= {HX} columns each")
    base, extra = divmod(lx, world)
    out, x0 = [], 0
    for r in range(world):
        w = base + (1 if r < extra else 0)
        out.append((x0, w))
        x0 += w
    return out


def slab_columns(lx: int, x0: int, w: int):
    """Global column of each of the w + 6 slab columns (halos wrap periodically)."""
    return [(x0 - HX + i) % lx for i in range(w + 2 * HX)]


class LatticeBackend:
    """The slab as a Lattice on this rank's GPU (the library's kernels)."""

    def __init__(self, lattice):
        self.lat = lattice
        self.w = lattice.lx - 2 * HX
        self.ly = lattice.ly

    def new_buffer(self, n):
        return torch.empty((37, self.ly, n), dtype=self.lat.dtype, device=self.lat.device)

    def current(self):
        return self.lat.state()

    def other(self):
        return self.lat.other()

    def swap(self):
        self.lat.swap()

    def pack(self, f, x0, n, buf):
        self.lat.pack_columns(f, x0, n, buf)

    def unpack(self, buf, x0, n, f):
        self.lat.unpack_columns(buf, x0, n, f)

    def step_columns(self, src, dst, x0, x1):
        if x1 > x0:
            self.lat.step_columns(src, dst, x0, x1)


class SlabRing:
    """pbc exchange and the bulk / border schedule of one rank's slab.

    rank, world: this rank in the ring (left = rank - 1, right = rank + 1,
    periodic); with world == 1 the slab is its own neighbour and the halos are
    refilled locally.  group: a torch.distributed process group (None = the
    default group).
    """

    def __init__(self, backend, rank: int = 0, world: int = 1, group=None):
        if backend.w < HX:
            raise ValueError(f"slab of {backend.w} columns: at least {HX} needed")
        self.b = backend
        self.rank, self.world, self.group = rank, world, group
        self.left = (rank - 1) % world
        self.right = (rank + 1) % world
        self.send_left = backend.new_buffer(HX)   # first physical columns -> left neighbour's right halo
        self.send_right = backend.new_buffer(HX)  # last physical columns -> right neighbour's left halo
        self.recv_left = backend.new_buffer(HX)   # into the left halo (from the left neighbour)
        self.recv_right = backend.new_buffer(HX)  # into the right halo (from the right neighbour)

    # ------------------------------------------------------------------
    def exchange_start(self, f):
        """Pack the border columns of state f and post the four messages."""
        w = self.b.w
        self.b.pack(f, HX, HX, self.send_left)
        self.b.pack(f, w, HX, self.send_right)
        if self.world == 1:
            return None
        import torch.distributed as dist
        # the same order on every rank: rightward flow, then leftward flow
        ops = [dist.P2POp(dist.isend, self.send_right, self._peer(self.right), self.group),
               dist.P2POp(dist.irecv, self.recv_left, self._peer(self.left), self.group),
               dist.P2POp(dist.isend, self.send_left, self._peer(self.left), self.group),
               dist.P2POp(dist.irecv, self.recv_right, self._peer(self.right), self.group)]
        return dist.batch_isend_irecv(ops)

    def exchange_finish(self, reqs, f):
        """Wait for the messages and write the halos of state f."""
        w = self.b.w
        if self.world == 1:
            self.b.unpack(self.send_right, 0, HX, f)
            self.b.unpack(self.send_left, w + HX, HX, f)
            return
        for r in reqs:
            r.wait()
        self.b.unpack(self.recv_left, 0, HX, f)
        self.b.unpack(self.recv_right, w + HX, HX, f)

    def _peer(self, r):
        if self.group is None:
            return r
        import torch.distributed as dist
        return dist.get_global_rank(self.group, r)

    # ------------------------------------------------------------------
    def bulk_and_border(self):
        """Column ranges [x0, x1) of the bulk (reads no halo column) and of the
        two borders (the three physical columns next to each halo)."""
        w = self.b.w
        lo, hi = HX, w + HX
        bulk = (2 * HX, w) if w > 2 * HX else (lo, lo)
        left = (lo, min(2 * HX, hi))
        right = (max(2 * HX, w), hi)
        return bulk, left, right

    def step(self, n: int = 1, overlap: bool = True):
        """n time steps: pbc, then propagate + bc + collide on the slab; with
        overlap the bulk is launched before the exchange completes and the
        borders after it (Fig. "schedulingop")."""
        bulk, left, right = self.bulk_and_border()
        for _ in range(n):
            src, dst = self.b.current(), self.b.other()
            reqs = self.exchange_start(src)
            if overlap:
                self.b.step_columns(src, dst, *bulk)
                self.exchange_finish(reqs, src)
                self.b.step_columns(src, dst, *left)
                self.b.step_columns(src, dst, *right)
            else:
                self.exchange_finish(reqs, src)
                self.b.step_columns(src, dst, HX, self.b.w + HX)
            self.b.swap()
        return self


def slab_lattice(lx: int, ly: int, rank: int, world: int, group=None, **lattice_kw):
    """This rank's slab of an lx x ly lattice as a Lattice on the current GPU
    and its SlabRing; returns (ring, x0, w).  lattice_kw go to Lattice
    (tau, g, t_top, t_bottom, precision, rho0).  The slab's lattice uses the
    current stream, the one torch.distributed orders its messages after."""
    from .lbm import Lattice
    x0, w = partition(lx, world)[rank]
    lat = Lattice(w + 2 * HX, ly, stream=torch.cuda.current_stream(), **lattice_kw)
    return SlabRing(LatticeBackend(lat), rank, world, group), x0, w
