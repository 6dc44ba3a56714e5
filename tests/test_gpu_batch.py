"""GPU parity of the batched, graph-captured multi-lattice step.

Every lattice of a batch of uneven sizes and parameters must evolve exactly
as the oracle evolves it alone (float64: <= 1e-12 per population plane;
float32 shifted storage: <= 2e-6 after one step), for every tile shape, and
the autotuner must leave a valid tile shape selected.
"""
import numpy as np
import pytest

import synth
from oracle import lattice, model as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1703_00186_gb300.batch import Batch

K = lattice.constants()

SPECS = [
    dict(lx=40, ly=24, tau=0.8, g=1e-3, delta=0.4),
    dict(lx=67, ly=45, tau=0.6, g=1e-4, delta=0.2),
    dict(lx=32, ly=6, tau=0.9, g=0.0, delta=0.6),
    dict(lx=100, ly=30, tau=0.7, g=5e-4, delta=0.3),
    dict(lx=3, ly=9, tau=1.0, g=2e-3, delta=0.5),
]


def fields(i, s):
    rho, ux, uy, T, tt, tb = synth.rt_fields(s["lx"], s["ly"], 2, 10 + i, delta=s["delta"], width=1.5)
    return (rho, ux, uy, T), tt, tb


def build(precision):
    specs = []
    flds = []
    for i, s in enumerate(SPECS):
        f, tt, tb = fields(i, s)
        specs.append(dict(lx=s["lx"], ly=s["ly"], tau=s["tau"], g=s["g"], t_top=tt, t_bottom=tb,
                          rho0=float(f[0].mean())))
        flds.append(f)
    return specs, flds


def plane_err(a, b):
    a, b = M.physical(a), M.physical(b)
    scale = np.abs(b).max(axis=(1, 2))
    return (np.abs(a - b).max(axis=(1, 2)) / scale).max()


def oracle_run(spec, f, n):
    p = M.Params(spec["lx"], spec["ly"], tau=spec["tau"], g=spec["g"], t_top=spec["t_top"],
                 t_bottom=spec["t_bottom"])
    return M.run(M.init_state(*f), p, n)


def test_tile_shapes():
    shapes = Batch.tile_shapes()
    assert len(shapes) == 13
    assert all(bx * by <= 256 and rows >= 1 for bx, by, rows in shapes)
    labels = Batch.tile_labels()
    assert labels[9] == "per-lattice 32x4" and not any(lb.startswith("per") for i, lb in enumerate(labels) if i != 9)
    assert labels[10:] == ["params 32x4x1", "params 32x4x4", "params 32x4x8"]


@pytest.mark.parametrize("tile", range(13))
def test_batch_fp64_matches_oracle_for_every_tile_shape(tile):
    specs, flds = build("fp64")
    b = Batch(specs, precision="fp64")
    b.set_tile(tile)
    for i, f in enumerate(flds):
        b.init(i, *f)
    n = 5
    b.step(2).step(3)   # two graph launches (cached graphs of 2 and 3 steps)
    for i, (s, f) in enumerate(zip(specs, flds)):
        got = b.state(i).cpu().numpy()
        assert plane_err(got, oracle_run(s, f, n)) <= 1e-12, i
    assert b.status() == 0


@pytest.mark.parametrize("tile", [0, 9, 10, 11, 12])
def test_batch_fp32_one_step_matches_oracle(tile):
    specs, flds = build("fp32")
    b = Batch(specs, precision="fp32")
    b.set_tile(tile)
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.step(1)
    for i, (s, f) in enumerate(zip(specs, flds)):
        rho0 = s["rho0"]
        d0 = (M.init_state(*f) - K["w"][:, None, None] * rho0).astype(np.float32)
        fin = d0.astype(np.float64) + K["w"][:, None, None] * rho0
        p = M.Params(s["lx"], s["ly"], tau=s["tau"], g=s["g"], t_top=s["t_top"], t_bottom=s["t_bottom"])
        want = M.step(fin, p)
        got = b.state(i).cpu().numpy().astype(np.float64) + K["w"][:, None, None] * rho0
        assert plane_err(got, want) <= 2e-6, i


def test_autotune_selects_a_valid_shape_and_results_stay_exact():
    specs, flds = build("fp64")
    b = Batch(specs, precision="fp64")
    for i, f in enumerate(flds):
        b.init(i, *f)
    best, times = b.autotune(steps=2)
    assert 0 <= best < len(Batch.tile_shapes())
    assert all(t > 0 for t in times) and times[best] == min(times)
    for i, f in enumerate(flds):   # the tuner advanced the lattices: start again
        b.init(i, *f)
    b.step(4)
    for i, (s, f) in enumerate(zip(specs, flds)):
        assert plane_err(b.state(i).cpu().numpy(), oracle_run(s, f, 4)) <= 1e-12


def test_batch_moments():
    specs, flds = build("fp64")
    b = Batch(specs, precision="fp64")
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.step(3)
    for i, (s, f) in enumerate(zip(specs, flds)):
        want = M.moments(M.physical(oracle_run(s, f, 3)))
        got = [t.cpu().numpy() for t in b.moments(i)]
        for g, w in zip(got, want):
            assert np.abs(g - w).max() <= 1e-12 * np.abs(w).max() + 1e-15


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_persistent_launch_matches_graph_launch(precision):
    specs, flds = build(precision)
    a = Batch(specs, precision=precision)
    b = Batch(specs, precision=precision)
    for i, f in enumerate(flds):
        a.init(i, *f)
        b.init(i, *f)
    a.step(5)
    b.step_persistent(2).step_persistent(3)
    assert b.status() == 0
    for i, s in enumerate(specs):
        np.testing.assert_array_equal(b.state(i).cpu().numpy()[:, 3:-3], a.state(i).cpu().numpy()[:, 3:-3])
        if precision == "fp64":
            assert plane_err(b.state(i).cpu().numpy(), oracle_run(s, flds[i], 5)) <= 1e-12


def test_bounded_barrier_wait_times_out_and_batch_stays_usable():
    from paper_1703_00186_gb300 import _lib as L
    specs, flds = build("fp64")
    b = Batch(specs, precision="fp64")
    assert b.barrier_selftest(20) == L.LBM_ERR_TIMEOUT   # the wait gave up, as designed
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.step_persistent(3)
    assert b.status() == 0
    for i, s in enumerate(specs):
        assert plane_err(b.state(i).cpu().numpy(), oracle_run(s, flds[i], 3)) <= 1e-12


@pytest.mark.parametrize("tile", [0, 1, 5, 8, 9])
def test_batch_fp64df_matches_oracle(tile):
    # float64 storage with the double-float collide, graph and persistent launches
    specs, flds = build("fp64df")
    b = Batch(specs, precision="fp64df")
    b.set_tile(tile)
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.step(2).step_persistent(2)
    assert b.status() == 0
    for i, (s, f) in enumerate(zip(specs, flds)):
        assert plane_err(b.state(i).cpu().numpy(), oracle_run(s, f, 4)) <= 1e-12, i


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-6), ("fp64df", 1e-13)])
def test_per_lattice_launches_match_the_batch_kernel(precision, tol):
    # candidate 9 steps each lattice with the single-lattice kernel on one of
    # eight streams: the batch kernel's arithmetic, compiled in another kernel
    # (float multiply-add contraction may differ), so the states agree to
    # rounding (odd and even step counts, two cached graphs)
    specs, flds = build(precision)
    a = Batch(specs, precision=precision)
    b = Batch(specs, precision=precision)
    a.set_tile(8)
    b.set_tile(9)
    for i, f in enumerate(flds):
        a.init(i, *f)
        b.init(i, *f)
    a.step(3).step(2)
    b.step(3).step(2)
    assert a.status() == 0 and b.status() == 0
    for i in range(len(specs)):
        sa, sb = a.state(i).cpu().numpy().astype(np.float64), b.state(i).cpu().numpy().astype(np.float64)
        if precision == "fp32":
            w = K["w"][:, None, None] * specs[i]["rho0"]
            sa, sb = sa + w, sb + w
        assert plane_err(sb, sa) <= tol, i


@pytest.mark.parametrize("tile", [10, 12])
def test_parameter_table_groups_match_per_lattice_launches(tile):
    # 70 lattices: two launches per step (groups of 64 and 6 lattices), each
    # lattice's constants read from the kernel-parameter table; against the
    # single-lattice kernel launched per lattice, to rounding
    rng = np.random.default_rng(5)
    specs, flds = [], []
    for i in range(70):
        lx, ly = int(rng.integers(3, 40)), int(rng.integers(6, 30))
        rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 2, 100 + i, delta=0.4, width=1.5)
        specs.append(dict(lx=lx, ly=ly, tau=float(rng.uniform(0.6, 1.0)), g=float(rng.uniform(0, 1e-3)),
                          t_top=tt, t_bottom=tb, rho0=float(rho.mean())))
        flds.append((rho, ux, uy, T))
    a = Batch(specs, precision="fp32")
    b = Batch(specs, precision="fp32")
    a.set_tile(9)
    b.set_tile(tile)
    for i, f in enumerate(flds):
        a.init(i, *f)
        b.init(i, *f)
    a.step(3)
    b.step(3)
    assert a.status() == 0 and b.status() == 0
    for i in range(len(specs)):
        w = K["w"][:, None, None] * specs[i]["rho0"]
        sa = a.state(i).cpu().numpy().astype(np.float64) + w
        sb = b.state(i).cpu().numpy().astype(np.float64) + w
        assert plane_err(sb, sa) <= 1e-6, i


def test_parameter_table_persistent_launch_matches_the_graph():
    # FP32 batch of at most 64 lattices: lbm_batch_step_persistent runs the
    # parameter-table kernel as one cooperative launch (L2-coherent loads,
    # bounded grid barrier); against the graph of the same kernel's tiles
    specs, flds = build("fp32")
    a = Batch(specs, precision="fp32")
    b = Batch(specs, precision="fp32")
    a.set_tile(12)
    for i, f in enumerate(flds):
        a.init(i, *f)
        b.init(i, *f)
    a.step(4)
    b.step_persistent(4)
    assert a.status() == 0 and b.status() == 0
    for i in range(len(specs)):
        w = K["w"][:, None, None] * specs[i]["rho0"]
        sa = a.state(i).cpu().numpy().astype(np.float64) + w
        sb = b.state(i).cpu().numpy().astype(np.float64) + w
        assert plane_err(sb, sa) <= 1e-6, i
