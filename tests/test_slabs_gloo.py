"""x-slab decomposition over ranks (Sect. 4, Fig. "schedulingop"), on CPU
ranks with the gloo backend.

Each rank steps its slab (w physical columns plus three halo columns on each
side) with the float64 oracle, and ``SlabRing`` - the exchange and schedule
the GPU path uses - refills the halos from the ring neighbours every step.
Assembled, the slabs must equal the oracle run on the whole lattice bit for
bit: every site's arithmetic is the same, only where its pull sources come
from differs.  Cases: two ranks (left and right neighbour are the same rank),
three ranks (a true ring) with uneven slabs, slabs narrower than six columns
(no bulk), and both schedules (bulk overlapping the exchange, and exchange
first).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import synth
from oracle import model as M
from paper_1703_00186_gb300.slabs import HX, SlabRing, partition, slab_columns


class OracleBackend:
    """A slab stepped by the float64 oracle on CPU tensors."""

    def __init__(self, p: M.Params, f0):
        self.p = p
        self.w = p.lx - 2 * HX
        self.ly = p.ly
        self.bufs = [torch.from_numpy(f0.copy()), torch.from_numpy(np.full_like(f0, np.nan))]
        self.cur = 0

    def new_buffer(self, n):
        return torch.empty((M.NPOP, self.ly, n), dtype=torch.float64)

    def current(self):
        return self.bufs[self.cur]

    def other(self):
        return self.bufs[1 - self.cur]

    def swap(self):
        self.cur ^= 1

    def pack(self, f, x0, n, buf):
        buf.copy_(f[:, HX:-HX, x0:x0 + n])

    def unpack(self, buf, x0, n, f):
        f[:, HX:-HX, x0:x0 + n] = buf

    def step_columns(self, src, dst, x0, x1):
        if x1 <= x0:
            return
        out = M.step(src.numpy(), self.p)
        dst[:, HX:-HX, x0:x1] = torch.from_numpy(out[:, HX:-HX, x0:x1])


def _case(lx, ly):
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 3, 5, delta=0.4)
    ux = 0.02 * synth.smooth_field(lx, ly, 6)
    p = M.Params(lx, ly, tau=0.7, g=1e-3, t_top=tt, t_bottom=tb)
    return p, (rho, ux, uy, T)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, lx, ly, steps, overlap, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, fields = _case(lx, ly)
        x0, w = partition(lx, world)[rank]
        cols = slab_columns(lx, x0, w)
        f0 = M.init_state(*[v[:, cols] for v in fields])
        f0[:, :, :HX] = np.nan  # the halos must come from the exchange
        f0[:, :, -HX:] = np.nan
        ps = M.Params(w + 2 * HX, ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom)
        ring = SlabRing(OracleBackend(ps, f0), rank, world)
        ring.step(steps, overlap=overlap)
        out[rank] = ring.b.current().numpy()[:, :, HX:w + HX].copy()
    finally:
        dist.destroy_process_group()


def _run_ranks(world, lx, ly, steps, overlap):
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, lx, ly, steps, overlap, out)) for r in range(world)]
    for pr in procs:
        pr.start()
    for pr in procs:
        pr.join(timeout=300)
        assert pr.exitcode == 0
    return np.concatenate([out[r] for r in range(world)], axis=2)


@pytest.mark.parametrize("world,lx,overlap", [(2, 23, True), (2, 23, False), (3, 17, True), (2, 10, True)])
def test_slabs_assemble_to_the_whole_lattice_bit_for_bit(world, lx, overlap):
    ly, steps = 12, 4
    got = _run_ranks(world, lx, ly, steps, overlap)
    p, fields = _case(lx, ly)
    want = M.run(M.init_state(*fields), p, steps)
    np.testing.assert_array_equal(M.physical(got), M.physical(want))


def test_partition_is_contiguous_ragged_and_refuses_thin_slabs():
    parts = partition(23, 3)
    assert parts == [(0, 8), (8, 8), (16, 7)]
    assert sum(w for _, w in parts) == 23
    assert slab_columns(23, 0, 8)[:HX] == [20, 21, 22] and slab_columns(23, 16, 7)[-HX:] == [0, 1, 2]
    with pytest.raises(ValueError):
        partition(8, 3)


def test_single_rank_ring_refills_its_own_halos_periodically():
    lx, ly, steps = 11, 12, 3
    p, fields = _case(lx, ly)
    cols = slab_columns(lx, 0, lx)
    f0 = M.init_state(*[v[:, cols] for v in fields])
    f0[:, :, :HX] = np.nan
    f0[:, :, -HX:] = np.nan
    ps = M.Params(lx + 2 * HX, ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom)
    ring = SlabRing(OracleBackend(ps, f0), 0, 1)
    ring.step(steps)
    got = ring.b.current().numpy()[:, :, HX:lx + HX]
    want = M.run(M.init_state(*fields), p, steps)
    np.testing.assert_array_equal(M.physical(got), M.physical(want))
