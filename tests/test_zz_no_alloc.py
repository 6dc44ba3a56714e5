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
each population plane's largest value).  It also checks that lam_out's halo
rows stay untouched and that a lattice wider than the array is refused.
"""
import ctypes

import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_adjoint_matches_context_adjoint_on_two_calls(precision):
    from paper_1703_00186_gb300 import _lib as L
    from paper_1703_00186_gb300.lbm import Lattice

    lib = L.load()
    lx, ly = 70, 37
    rho, ux, uy, T = synth.random_fields(lx, ly, 90, umax=0.08)
    lat = Lattice(lx, ly, tau=0.7, g=1e-3, t_top=0.85, t_bottom=1.2, precision=precision, rho0=1.0)
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


def test_noalloc_adjoint_refuses_lattices_wider_than_its_array():
    from paper_1703_00186_gb300 import _lib as L

    lib = L.load()
    big = L.LbmParams(L.LBM_NOALLOC_MAX_LX + 1, 8, L.LBM_FP64, 0, 0.8, 0.0, 1.0, 1.0, 1.0)
    rc = lib.lbm_adjoint_step_noalloc(ctypes.byref(big), ctypes.c_void_p(256), ctypes.c_void_p(512),
                                      ctypes.c_void_p(1024), None)
    assert rc == L.LBM_ERR_SIZE
