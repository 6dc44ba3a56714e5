"""Parity at the benchmark's full sizes, in the launch configuration it times.

The GPU steps the whole lattice; the oracle reproduces sampled outputs.  An
output column after n steps depends only on input columns within 3 n of it
(propagate pulls from at most 3 sites away; the wall sums gather from the
same neighbourhood), so the oracle runs on periodic column windows cut from
the same seeded fields, widened by 3 n + 3 columns on each side, and its
interior columns are compared with the GPU's.  Every window spans the full
height, so both walls are included; one window crosses the periodic seam.

Tolerances as in test_gpu_parity.py: float64 paths 1e-12 per population
plane of the window, float32 shifted storage 2e-6.
"""
import numpy as np
import pytest

import synth
from oracle import lattice, model as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1703_00186_gb300.batch import Batch
    from paper_1703_00186_gb300.lbm import Lattice

K = lattice.constants()
LX, LY = 2048, 4096


def window_run(fields, p, x0, w, n, encode_rho0=None):
    """Oracle state after n steps on columns [x0, x0 + w) (periodic in x)."""
    pad = 3 * n + 3
    cols = (x0 - pad + np.arange(w + 2 * pad)) % p.lx
    sub = [np.ascontiguousarray(a[:, cols]) for a in fields]
    q = M.Params(len(cols), p.ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom)
    f = M.init_state(*sub)
    if encode_rho0 is not None:   # the float32 path starts from the float32 encoding
        f[:, 3:-3] = (f[:, 3:-3] - K["w"][:, None, None] * encode_rho0).astype(np.float32) \
            .astype(np.float64) + K["w"][:, None, None] * encode_rho0
    f = M.run(f, q, n)
    return M.physical(f)[:, :, pad:pad + w]


def window_err(gpu_state, want, x0, w, lx, rho0=None):
    cols = (x0 + np.arange(w)) % lx
    got = gpu_state[:, 3:-3][:, :, cols]
    if rho0 is not None:
        got = got.astype(np.float64) + K["w"][:, None, None] * rho0
    scale = np.abs(want).max(axis=(1, 2))
    return (np.abs(got - want).max(axis=(1, 2)) / scale).max()


WINDOWS = [(0, 12), (1017, 16), (2040, 8)]   # the last one crosses the seam


@pytest.fixture(scope="module")
def rt():
    rho, ux, uy, T, tt, tb = synth.rt_fields(LX, LY, 32, 0)
    p = M.Params(LX, LY, tau=0.6, g=1e-5, t_top=tt, t_bottom=tb)
    return (rho, ux, uy, T), p


@pytest.mark.parametrize("precision", ["fp64", "fp64df"])
def test_full_size_float64_paths_on_sampled_columns(rt, precision):
    fields, p = rt
    n = 2
    lat = Lattice(LX, LY, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom, precision=precision)
    lat.init(*fields).step(n)
    state = lat.state().cpu().numpy()
    for x0, w in WINDOWS:
        want = window_run(fields, p, x0, w, n)
        assert window_err(state, want, x0, w, LX) <= 1e-12, (x0, w)


def test_full_size_fp32_store_on_sampled_columns(rt):
    fields, p = rt
    rho0 = float(fields[0].mean())
    lat = Lattice(LX, LY, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom, precision="fp32", rho0=rho0)
    lat.init(*fields).step(1)
    state = lat.state().cpu().numpy()
    for x0, w in WINDOWS:
        want = window_run(fields, p, x0, w, 1, encode_rho0=rho0)
        assert window_err(state, want, x0, w, LX, rho0=rho0) <= 2e-6, (x0, w)


def test_full_64_lattice_batch_on_sampled_lattices():
    specs = synth.batch_lattices(64, 7)
    flds, descs = [], []
    for sp in specs:
        rho, ux, uy, T, tt, tb = synth.rt_fields(sp.lx, sp.ly, 8, sp.seed, delta=sp.delta)
        flds.append((rho, ux, uy, T))
        descs.append(dict(lx=sp.lx, ly=sp.ly, tau=sp.tau, g=sp.g, t_top=tt, t_bottom=tb, rho0=float(rho.mean())))
    b = Batch(descs, precision="fp32")
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.autotune(steps=1)
    for i, f in enumerate(flds):
        b.init(i, *f)
    b.step(1)
    sizes = [d["lx"] * d["ly"] for d in descs]
    for i in sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17}):
        d = descs[i]
        p = M.Params(d["lx"], d["ly"], tau=d["tau"], g=d["g"], t_top=d["t_top"], t_bottom=d["t_bottom"])
        state = b.state(i).cpu().numpy()
        for x0, w in ((0, 8), (d["lx"] // 2, 8)):
            want = window_run(flds[i], p, x0, w, 1, encode_rho0=d["rho0"])
            assert window_err(state, want, x0, w, d["lx"], rho0=d["rho0"]) <= 2e-6, (i, x0)


def test_adjoint_step_at_rollout_size_on_sampled_columns():
    # the 256 x 512 lattice of the checkpointed-rollout benchmark
    from oracle import adjoint as A
    lx, ly = 256, 512
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 4, 1)
    p = M.Params(lx, ly, tau=0.8, g=1e-4, t_top=tt, t_bottom=tb)
    lam = np.full((37, ly + 6, lx), np.nan)
    lam[:, 3:-3] = synth.noise(lx, ly, 77)
    lat = Lattice(lx, ly, tau=p.tau, g=p.g, t_top=tt, t_bottom=tb)
    lat.init(rho, ux, uy, T)
    got = lat.adjoint_step(lat.state(), torch.as_tensor(lam, device="cuda")).cpu().numpy()
    pad = 9
    for x0, w in ((0, 8), (131, 8), (250, 8)):
        cols = (x0 - pad + np.arange(w + 2 * pad)) % lx
        q = M.Params(len(cols), ly, tau=p.tau, g=p.g, t_top=tt, t_bottom=tb)
        f_t = M.init_state(*[np.ascontiguousarray(a[:, cols]) for a in (rho, ux, uy, T)])
        want = M.physical(A.adjoint_step(f_t, np.ascontiguousarray(lam[:, :, cols]), q))[:, :, pad:pad + w]
        g = got[:, 3:-3][:, :, (x0 + np.arange(w)) % lx]
        scale = np.abs(want).max(axis=(1, 2))
        assert (np.abs(g - want).max(axis=(1, 2)) / scale).max() <= 1e-12, x0
