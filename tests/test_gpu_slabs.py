"""The x-slab path of the library on one GPU (Sect. 4, Fig. "schedulingop").

* lbm_step_columns over column ranges that tile the lattice gives the full
  step bit for bit (the bulk / border split changes no site's arithmetic);
* lbm_pack_columns / lbm_unpack_columns move exactly the named columns;
* one slab that is its own ring neighbour (SlabRing, world = 1) steps like the
  periodic lattice, bit for bit, with and without the overlapped schedule;
* three slabs on this one GPU, their halos refilled from each other through
  the pack / unpack kernels every step, assemble to the single-lattice run
  bit for bit.  (The slabs are stepped one after the other: no kernel waits
  for another.  The exchange between processes is covered by the gloo tests
  on CPU; NCCL between GPUs is not run here: one GPU.)
"""
import numpy as np
import pytest

import synth
from oracle import model as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1703_00186_gb300 import _lib as L
    from paper_1703_00186_gb300.lbm import Lattice
    from paper_1703_00186_gb300.slabs import HX, LatticeBackend, SlabRing, partition, slab_columns


def fields(lx, ly, seed=5):
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 3, seed, delta=0.4)
    ux = 0.02 * synth.smooth_field(lx, ly, 6)
    return (rho, ux, uy, T), dict(tau=0.7, g=1e-3, t_top=tt, t_bottom=tb)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_column_ranges_tile_the_full_step(precision):
    lx, ly = 70, 24
    flds, kw = fields(lx, ly)
    lat = Lattice(lx, ly, precision=precision, rho0=1.0, **kw).init(*flds)
    src = lat.state()
    want = lat.step_from(src, lat.new_state())
    got = lat.new_state()
    for x0, x1 in ((0, 3), (3, 40), (40, 40), (40, 67), (67, 70)):
        lat.step_columns(src, got, x0, x1)
    assert torch.equal(M.physical(got), M.physical(want))


def test_pack_and_unpack_move_exactly_the_named_columns():
    lx, ly = 40, 12
    flds, kw = fields(lx, ly)
    lat = Lattice(lx, ly, **kw).init(*flds).step(2)
    f = lat.state()
    buf = torch.empty((37, ly, 5), dtype=torch.float64, device="cuda")
    lat.pack_columns(f, 30, 5, buf)
    assert torch.equal(buf, f[:, HX:-HX, 30:35])
    g = torch.full_like(f, float("nan"))
    lat.unpack_columns(buf, 2, 5, g)
    assert torch.equal(g[:, HX:-HX, 2:7], buf)
    assert torch.isnan(g[:, :, :2]).all() and torch.isnan(g[:, :, 7:]).all() and torch.isnan(g[:, :HX]).all()
    with pytest.raises(L.LBMError):
        lat.step_columns(f, g, 5, 41)
    with pytest.raises(L.LBMError):
        lat.pack_columns(f, 38, 3, torch.empty((37, ly, 3), dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("precision,overlap", [("fp64", True), ("fp64", False), ("fp32", True)])
def test_single_slab_ring_equals_the_periodic_lattice(precision, overlap):
    lx, ly, steps = 45, 20, 6
    flds, kw = fields(lx, ly)
    ref = Lattice(lx, ly, precision=precision, rho0=1.0, **kw).init(*flds).step(steps)
    cols = slab_columns(lx, 0, lx)
    slab = Lattice(lx + 2 * HX, ly, precision=precision, rho0=1.0, stream=torch.cuda.current_stream(), **kw)
    slab.init(*[v[:, cols] for v in flds])
    ring = SlabRing(LatticeBackend(slab), 0, 1)
    ring.step(steps, overlap=overlap)
    assert torch.equal(M.physical(slab.state())[:, :, HX:lx + HX], M.physical(ref.state()))


def test_three_slabs_on_one_gpu_assemble_to_the_single_lattice():
    lx, ly, steps = 53, 18, 5
    flds, kw = fields(lx, ly)
    ref = Lattice(lx, ly, **kw).init(*flds).step(steps)
    slabs = []
    for x0, w in partition(lx, 3):
        lat = Lattice(w + 2 * HX, ly, **kw)
        lat.init(*[v[:, slab_columns(lx, x0, w)] for v in flds])
        ring = SlabRing(LatticeBackend(lat), 0, 1)   # its buffers and schedule; the exchange is done below
        slabs.append((lat, ring, w))
    n = len(slabs)
    for _ in range(steps):
        for lat, ring, w in slabs:
            lat.pack_columns(lat.state(), HX, HX, ring.send_left)
            lat.pack_columns(lat.state(), w, HX, ring.send_right)
        for i, (lat, ring, w) in enumerate(slabs):
            lat.unpack_columns(slabs[(i - 1) % n][1].send_right, 0, HX, lat.state())
            lat.unpack_columns(slabs[(i + 1) % n][1].send_left, w + HX, HX, lat.state())
        for lat, ring, w in slabs:
            bulk, left, right = ring.bulk_and_border()
            src, dst = lat.state(), lat.other()
            for x0, x1 in (bulk, left, right):
                if x1 > x0:
                    lat.step_columns(src, dst, x0, x1)
            lat.swap()
    got = torch.cat([M.physical(lat.state())[:, :, HX:w + HX] for lat, _, w in slabs], dim=2)
    assert torch.equal(got, M.physical(ref.state()))
