"""The adjoint step for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc.  Their device memory may all be owned by
another allocator (for example a framework's caching allocator that reserved
the GPU up front).  Or they must not allocate after their set-up phase,
because cudaMalloc can synchronise the device.  Such callers cannot create a
context, since creating one allocates a small device block.  For them the
library offers lbm_adjoint_step_noalloc: no context, no allocation, and its
scratch is a fixed array inside the library.

This test calls that entry point through the C ABI twice in a row, with
different cotangents.  It checks each result against the context entry point
lbm_adjoint_step on the same inputs, within the adjoint tolerance (1e-12 of
each population plane's largest value), for every precision, for a lattice
wider than one block of the wall kernel and for a periodic-y lattice (no
walls, so the fixed array is not used).  It checks one call directly against
the oracle's adjoint step, that lam_out's halo rows stay untouched, and that a
lattice wider than the array is refused with nothing written.
"""
import ctypes

import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("precision,lx,ly,periodic_y", [
    ("fp64", 70, 37, False), ("fp32", 70, 37, False), ("fp64df", 70, 37, False),
    ("fp64", 300, 12, False), ("fp64", 40, 24, True)])
def test_noalloc_adjoint_matches_context_adjoint_on_two_calls(precision, lx, ly, periodic_y):
    from paper_1703_00186_gb300 import _lib as L
    from paper_1703_00186_gb300.lbm import Lattice

    lib = L.load()
    rho, ux, uy, T = synth.random_fields(lx, ly, 90, umax=0.08)
    lat = Lattice(lx, ly, tau=0.7, g=1e-3, t_top=0.85, t_bottom=1.2, precision=precision, rho0=1.0,
                  periodic_y=periodic_y)
    lat.init(rho, ux, uy, T).step(3)
    f_t = lat.state().clone()
    gen = torch.Generator(device="cuda").manual_seed(91)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        lam_in = torch.randn(lat.shape, dtype=torch.float64, device="cuda", generator=gen)
        want = lat.adjoint_step(f_t, lam_in)
        got = torch.full(lat.shape, float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.lbm_adjoint_step_noalloc(ctypes.byref(lat.params), _ptr(f_t), _ptr(lam_in), _ptr(got), stream)
        assert rc == L.LBM_OK
        torch.cuda.synchronize()
        g, w = got[:, 3:-3], want[:, 3:-3]
        err = ((g - w).abs().amax(dim=(1, 2)) / w.abs().amax(dim=(1, 2))).max().item()
        assert err <= 1e-12, err
        assert torch.isnan(got[:, :3]).all() and torch.isnan(got[:, -3:]).all()


def test_noalloc_adjoint_matches_the_oracle_adjoint():
    import numpy as np

    from oracle import adjoint as A, model as M
    from paper_1703_00186_gb300 import _lib as L
    from paper_1703_00186_gb300.lbm import Lattice

    lib = L.load()
    lx, ly = 20, 12
    p = M.Params(lx, ly, tau=0.7, g=1e-3, t_top=0.85, t_bottom=1.2)
    rho, ux, uy, T = synth.random_fields(lx, ly, 92, umax=0.08)
    f = M.run(M.init_state(rho, ux, uy, T), p, 2)
    lam = np.random.default_rng(93).standard_normal(f.shape)
    want = M.physical(A.adjoint_step(f, lam, p))
    lat = Lattice(lx, ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom)
    f_t = torch.as_tensor(f, device="cuda")
    lam_in = torch.as_tensor(lam, device="cuda")
    got = torch.full(lat.shape, float("nan"), dtype=torch.float64, device="cuda")
    rc = lib.lbm_adjoint_step_noalloc(ctypes.byref(lat.params), _ptr(f_t), _ptr(lam_in), _ptr(got),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.LBM_OK
    g = M.physical(got.cpu().numpy())
    err = (np.abs(g - want).max(axis=(1, 2)) / np.abs(want).max(axis=(1, 2))).max()
    assert err <= 1e-12, err


def test_noalloc_adjoint_refuses_lattices_wider_than_its_array():
    # Buffers of the right size for the refused lattice, so that even a
    # launch would stay inside them; the call must write nothing.
    from paper_1703_00186_gb300 import _lib as L

    lib = L.load()
    lx, ly = L.LBM_NOALLOC_MAX_LX + 1, 8
    big = L.LbmParams(lx, ly, L.LBM_FP64, 0, 0.8, 0.0, 1.0, 1.0, 1.0)
    shape = (37, ly + 6, lx)
    f_t = torch.zeros(shape, dtype=torch.float64, device="cuda")
    lam_in = torch.zeros(shape, dtype=torch.float64, device="cuda")
    lam_out = torch.full(shape, 7.0, dtype=torch.float64, device="cuda")
    rc = lib.lbm_adjoint_step_noalloc(ctypes.byref(big), _ptr(f_t), _ptr(lam_in), _ptr(lam_out),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.LBM_ERR_SIZE
    torch.cuda.synchronize()
    assert bool((lam_out == 7.0).all())
