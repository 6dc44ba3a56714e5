"""GPU parity of the discrete adjoint kernels against the oracle's adjoint.

The oracle forms the collide Jacobian by complex-step derivatives and writes
(B P)^T out by hand; the kernels use analytic derivatives of the Hermite
polynomial.  Tolerance: max |gpu - oracle| <= 1e-12 times max |oracle| per
population plane (float64 on both sides, different association).
"""
import numpy as np
import pytest

import synth
from oracle import adjoint as A, lattice, model as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1703_00186_gb300.lbm import Lattice

K = lattice.constants()


def to_dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def noisy_state(lx, ly, seed, eps=0.03):
    rho, ux, uy, T = synth.random_fields(lx, ly, seed, umax=0.08)
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] *= 1.0 + eps * synth.noise(lx, ly, seed + 1)
    return f


def rand_cot(lx, ly, seed):
    lam = np.full((37, ly + 6, lx), np.nan)
    lam[:, 3:-3] = np.random.default_rng(seed).standard_normal((37, ly, lx))
    return lam


def plane_err(a, b):
    a, b = M.physical(a), M.physical(b)
    scale = np.abs(b).max(axis=(1, 2))
    return (np.abs(a - b).max(axis=(1, 2)) / scale).max()


def make(p, precision="fp64", rho0=1.0):
    return Lattice(p.lx, p.ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom,
                   precision=precision, rho0=rho0, periodic_y=p.periodic_y)


@pytest.mark.parametrize("lx,ly", [(13, 10), (35, 7), (3, 6)])
@pytest.mark.parametrize("periodic_y", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "fp64df"])
def test_adjoint_step_parity(lx, ly, periodic_y, precision):
    # fp64df: the cotangent sums run in double-float (about 48 bits); the
    # float64 bar holds for them too
    p = M.Params(lx, ly, tau=0.7, g=2e-3, t_top=0.85, t_bottom=1.2, periodic_y=periodic_y)
    f = noisy_state(lx, ly, 40 + lx)
    lam = rand_cot(lx, ly, 41 + ly)
    want = A.adjoint_step(f, lam, p)
    lat = make(p, precision=precision)
    got = lat.adjoint_step(to_dev(f), to_dev(lam)).cpu().numpy()
    assert plane_err(got, want) <= 1e-12


@pytest.mark.parametrize("scale", [1e-200, 1e-30, 3.0, 1e150, 1e300, 1e-300])
def test_adjoint_step_parity_at_any_cotangent_scale(scale):
    # The float64 kernel sums the cotangents in block-scaled fixed point (one
    # exponent per site): 1e300 sits near the top of its range, 1e-300 below
    # it (those sites take the float64 sums).  Every scale meets the float64
    # bar, and a power-of-two scale of the cotangents scales the result
    # exactly.
    lx, ly = 21, 9
    p = M.Params(lx, ly, tau=0.7, g=2e-3, t_top=0.85, t_bottom=1.2)
    f = noisy_state(lx, ly, 60)
    lam = rand_cot(lx, ly, 61) * scale
    lam[:, 3:-3][5, 4, 7] = 0.0                      # zero cotangents are exact
    lam[:, 3:-3][:, 2, 3] = 0.0                      # a site with no cotangent at all
    want = A.adjoint_step(f, lam, p)
    lat = make(p)
    got = lat.adjoint_step(to_dev(f), to_dev(lam)).cpu().numpy()
    assert np.isfinite(M.physical(got)).all()
    assert plane_err(got, want) <= 1e-12
    if 1e-250 < scale < 1e250:                       # fixed-point path before and after
        halved = lat.adjoint_step(to_dev(f), to_dev(lam * 2.0 ** -40)).cpu().numpy()
        np.testing.assert_array_equal(M.physical(halved), M.physical(got) * 2.0 ** -40)


def test_adjoint_step_fp32_state_parity():
    lx, ly = 16, 12
    rho0 = 1.05
    p = M.Params(lx, ly, tau=0.75, g=1e-3, t_top=0.9, t_bottom=1.1)
    f = noisy_state(lx, ly, 50)
    d = (f - K["w"][:, None, None] * rho0).astype(np.float32)
    fdec = d.astype(np.float64) + K["w"][:, None, None] * rho0
    lam = rand_cot(lx, ly, 51)
    want = A.adjoint_step(fdec, lam, p)
    lat = make(p, precision="fp32", rho0=rho0)
    got = lat.adjoint_step(to_dev(d, torch.float32), to_dev(lam)).cpu().numpy()
    assert plane_err(got, want) <= 1e-12


def test_moments_vjp_parity():
    lx, ly = 21, 9
    p = M.Params(lx, ly, tau=0.8)
    f = noisy_state(lx, ly, 60)
    rng = np.random.default_rng(61)
    g = [rng.standard_normal((ly, lx)) for _ in range(4)]
    want = A.moments_vjp(f, *g)
    lat = make(p)
    got = lat.moments_vjp(to_dev(f), *g).cpu().numpy()
    assert plane_err(got, want) <= 1e-12
    # a NULL cotangent field counts as zero
    want_t = A.moments_vjp(f, 0 * g[0], 0 * g[0], 0 * g[0], g[3])
    got_t = lat.moments_vjp(to_dev(f), None, None, None, g[3]).cpu().numpy()
    assert plane_err(got_t, want_t) <= 1e-12


def test_init_vjp_parity():
    lx, ly = 19, 11
    p = M.Params(lx, ly, tau=0.8)
    rho, ux, uy, T = synth.random_fields(lx, ly, 70, umax=0.1)
    lam = rand_cot(lx, ly, 71)
    want = A.equilibrium_vjp(rho, ux, uy, T, lam)
    lat = make(p)
    got = [t.cpu().numpy() for t in lat.init_vjp(rho, ux, uy, T, to_dev(lam))]
    for g, w in zip(got, want):
        assert np.abs(g - w).max() <= 1e-12 * np.abs(w).max()


def test_moments_vjp_fp32_state_parity():
    lx, ly = 21, 9
    rho0 = 1.05
    p = M.Params(lx, ly, tau=0.8)
    f = noisy_state(lx, ly, 62)
    d = (f - K["w"][:, None, None] * rho0).astype(np.float32)
    fdec = d.astype(np.float64) + K["w"][:, None, None] * rho0
    rng = np.random.default_rng(63)
    g = [rng.standard_normal((ly, lx)) for _ in range(4)]
    want = A.moments_vjp(fdec, *g)
    lat = make(p, precision="fp32", rho0=rho0)
    got = lat.moments_vjp(to_dev(d, torch.float32), *g).cpu().numpy()
    assert plane_err(got, want) <= 1e-12


# ---------------------------------------------------------------------------
# Float32 cotangents (lbm_adjoint_step_f32, FP32-store lattices).  Every
# cotangent sum and the relaxation run in float32: each result carries a few
# float32 roundings (unit 6e-8) of terms up to about 10 times the plane's
# largest value, so the bar is 2e-6 of the plane's max |oracle| (measured
# 2-4e-7).  The oracle takes the float32 cotangents exactly (as float64).

@pytest.mark.parametrize("lx,ly,periodic_y", [(16, 12, False), (35, 7, True), (40, 24, False)])
def test_adjoint_step_f32_parity(lx, ly, periodic_y):
    rho0 = 1.05
    p = M.Params(lx, ly, tau=0.75, g=1e-3, t_top=0.9, t_bottom=1.1, periodic_y=periodic_y)
    f = noisy_state(lx, ly, 70 + lx)
    d = (f - K["w"][:, None, None] * rho0).astype(np.float32)
    fdec = d.astype(np.float64) + K["w"][:, None, None] * rho0
    lam32 = rand_cot(lx, ly, 71 + ly).astype(np.float32)
    want = A.adjoint_step(fdec, lam32.astype(np.float64), p)
    lat = make(p, precision="fp32", rho0=rho0)
    got = lat.adjoint_step(to_dev(d, torch.float32), to_dev(lam32, torch.float32))
    assert got.dtype == torch.float32
    assert plane_err(got.cpu().numpy().astype(np.float64), want) <= 2e-6


def test_adjoint_step_f32_is_for_fp32_store_lattices_only():
    from paper_1703_00186_gb300._lib import LBMError
    p = M.Params(16, 12, tau=0.8)
    lat = make(p)
    f = to_dev(noisy_state(16, 12, 80))
    lam = to_dev(rand_cot(16, 12, 81), torch.float32)
    with pytest.raises(LBMError):
        lat.adjoint_step(f, lam)


def test_moments_and_init_vjp_with_float32_cotangents():
    # computed in float64 and rounded once (moments), or read from float32
    # (init): the float32 rounding of the cotangents is the only difference
    lx, ly = 21, 9
    rho0 = 1.05
    p = M.Params(lx, ly, tau=0.8)
    f = noisy_state(lx, ly, 90)
    d = (f - K["w"][:, None, None] * rho0).astype(np.float32)
    fdec = d.astype(np.float64) + K["w"][:, None, None] * rho0
    g = [np.random.default_rng(91 + i).standard_normal((ly, lx)) for i in range(4)]
    lat = make(p, precision="fp32", rho0=rho0)
    got = lat.moments_vjp(to_dev(d, torch.float32), *g, dtype=torch.float32)
    assert got.dtype == torch.float32
    want = A.moments_vjp(fdec, *g)
    assert plane_err(got.cpu().numpy().astype(np.float64), want) <= 1e-7
    rho, ux, uy, T = synth.random_fields(lx, ly, 92, umax=0.1)
    lam32 = rand_cot(lx, ly, 93).astype(np.float32)
    gq = [t.cpu().numpy() for t in lat.init_vjp(rho, ux, uy, T, to_dev(lam32, torch.float32))]
    wq = A.equilibrium_vjp(rho, ux, uy, T, lam32.astype(np.float64))
    for a, b in zip(gq, wq):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
