"""GPU parity of the fused D2Q37 step against the float64 oracle.

Tolerances:
* propagate + bc (pure moves, fixed-order wall sums, one product): bit-exact;
* float64 full step: max |gpu - oracle| per population plane <= 1e-12 times
  the plane's max |oracle| (the kernels evaluate the same polynomial with a
  different association and FMA, so rounding differs at ~1e-16 per step);
* float32 shifted storage: <= 2e-6 relative after 1 step, checked against
  the float64 oracle (float32 rounding of the stored deviations).
"""
import numpy as np
import pytest

import synth
from oracle import lattice, model as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1703_00186_gb300.lbm import Lattice

K = lattice.constants()


def to_dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def encode32(f, rho0):
    return (f - K["w"][:, None, None] * rho0).astype(np.float32)


def decode32(d, rho0):
    return d.astype(np.float64) + K["w"][:, None, None] * rho0


def noisy_state(lx, ly, seed, eps=0.02, umax=0.1):
    rho, ux, uy, T = synth.random_fields(lx, ly, seed, umax=umax)
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] *= 1.0 + eps * synth.noise(lx, ly, seed + 1)
    return f


def plane_err(a, b):
    a, b = M.physical(a), M.physical(b)
    scale = np.abs(b).max(axis=(1, 2))
    return (np.abs(a - b).max(axis=(1, 2)) / scale).max()


def make(p: M.Params, precision="fp64", rho0=1.0):
    return Lattice(p.lx, p.ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom,
                   precision=precision, rho0=rho0, periodic_y=p.periodic_y)


def test_library_constants_are_bit_identical_to_oracle():
    p = M.Params(16, 12, tau=0.8, t_top=0.5, t_bottom=1.5)
    lat = make(p)
    r, w, qb, qt = lat.constants()
    assert r == K["r"]
    np.testing.assert_array_equal(w, K["w"])
    np.testing.assert_array_equal(qb, M.wall_q(1.5, "bottom"))
    np.testing.assert_array_equal(qt, M.wall_q(0.5, "top"))


@pytest.mark.parametrize("lx,ly", [(64, 128), (67, 45), (3, 6), (130, 9)])
@pytest.mark.parametrize("periodic_y", [False, True])
def test_propagate_bc_is_bit_exact(lx, ly, periodic_y):
    p = M.Params(lx, ly, tau=0.8, g=1e-4, t_top=0.7, t_bottom=1.3, periodic_y=periodic_y)
    f = noisy_state(lx, ly, 100 + lx + ly, eps=0.3)
    f[:, :3] = np.nan          # halos are never read as data
    f[:, -3:] = np.nan
    want = M.propagate_bc(f, p)
    lat = make(p)
    got = lat.propagate_bc(to_dev(f)).cpu().numpy()
    np.testing.assert_array_equal(M.physical(got), M.physical(want))


def test_init_matches_oracle_equilibrium():
    lx, ly = 40, 24
    rho, ux, uy, T = synth.random_fields(lx, ly, 7)
    p = M.Params(lx, ly, tau=0.8)
    lat = make(p)
    lat.init(rho, ux, uy, T)
    got = lat.state().cpu().numpy()
    assert plane_err(got, M.init_state(rho, ux, uy, T)) < 1e-14


@pytest.mark.parametrize("lx,ly", [(64, 128), (67, 45), (3, 6)])
@pytest.mark.parametrize("periodic_y", [False, True])
def test_one_step_parity_fp64(lx, ly, periodic_y):
    p = M.Params(lx, ly, tau=0.7, g=2e-3, t_top=0.8, t_bottom=1.2, periodic_y=periodic_y)
    f = noisy_state(lx, ly, 200 + lx, eps=0.05)
    want = M.step(f, p)
    lat = make(p)
    lat.set_state(to_dev(f))
    lat.step(1)
    got = lat.state().cpu().numpy()
    assert np.isnan(got[:, :3]).all() and np.isnan(got[:, -3:]).all()  # halos untouched
    assert plane_err(got, want) <= 1e-12


def test_rayleigh_taylor_64x128_100_steps_fp64():
    # 64 x 128, 4 interface modes, tau = 0.8, g = 1e-4, 100 steps
    rho, ux, uy, T, tt, tb = synth.rt_fields(64, 128, 4, 0)
    p = M.Params(64, 128, tau=0.8, g=1e-4, t_top=tt, t_bottom=tb)
    f0 = M.init_state(rho, ux, uy, T)
    lat = make(p)
    lat.init(rho, ux, uy, T)
    g1 = lat.state().cpu().numpy()
    assert plane_err(g1, f0) < 1e-14
    lat.set_state(to_dev(f0))
    want = f0
    for n in (1, 99):
        lat.step(n)
        want = M.run(want, p, n)
        got = lat.state().cpu().numpy()
        assert plane_err(got, want) <= 1e-12, n
    fields = [t.cpu().numpy() for t in lat.moments()]
    ref = M.moments(M.physical(want))
    for g, r in zip(fields, ref):
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max() + 1e-15


def test_moment_sums_are_the_correctly_rounded_exact_sums():
    # The float64 moment sums are formed exactly (fixed point on the integer
    # pipe) and rounded once: rho must equal the exact rational sum of the
    # stored populations rounded to nearest, bit for bit, for populations of
    # mixed signs and magnitudes (all >= 2^-30, so nothing is truncated), and
    # for a site holding a population outside the fixed-point range (|f| >= 4,
    # float64 fallback) it must still be within float64 rounding.
    from fractions import Fraction
    lx, ly = 19, 7
    rng = np.random.default_rng(93)
    f = noisy_state(lx, ly, 92, eps=0.05)
    phys = f[:, 3:-3]
    phys *= np.where(rng.random(phys.shape) < 0.1, -1.0, 1.0)          # some negative populations
    phys *= 2.0 ** rng.integers(-20, 3, phys.shape)                       # spread of exponents
    small = (np.abs(phys) < 2.0 ** -30) & (phys != 0)
    phys[small] = np.copysign(2.0 ** -30, phys[small])
    phys[rng.random(phys.shape) < 0.02] = 0.0
    phys[:, 2, 5] = 3.999999                                              # top of the exact range
    phys[7, 4, 11] = 5.0                                                  # outside: float64 fallback
    lat = make(M.Params(lx, ly, tau=0.8))
    rho = lat.moments(to_dev(f))[0].cpu().numpy()
    for y in range(ly):
        for x in range(lx):
            exact = sum(Fraction(float(v)) for v in phys[:, y, x])
            if (y, x) == (4, 11):
                assert abs(rho[y, x] - float(exact)) <= 1e-14 * np.abs(phys[:, y, x]).sum()
            else:
                assert rho[y, x] == float(exact), (y, x)


def test_moment_sums_with_tiny_and_zero_populations():
    # Populations below 2^-30 keep their bits down to 2^-82 only, so a sum with
    # such terms is within one unit in the last place of the exact sum (the
    # rounding may fall on either side of a tie); signed zeros and values at the
    # bottom of the float64 range are handled without a fallback.
    from fractions import Fraction
    lx, ly = 8, 6
    f = noisy_state(lx, ly, 94, eps=0.05)
    phys = f[:, 3:-3]
    tiny = [1e-300, -1e-300, 2.0 ** -60, -(2.0 ** -45), 1e-20, 0.0, -0.0, 3e-12]
    for i, v in enumerate(tiny):
        phys[5 + i, i % ly, (3 * i) % lx] = v
    phys[:, 0, 0] = 0.0
    phys[0, 0, 0] = 2.0 ** -70                                            # a site of tiny mass
    lat = make(M.Params(lx, ly, tau=0.8))
    rho = lat.moments(to_dev(f))[0].cpu().numpy()
    for y in range(ly):
        for x in range(lx):
            exact = float(sum(Fraction(float(v)) for v in phys[:, y, x]))
            assert abs(rho[y, x] - exact) <= np.spacing(abs(exact)), (y, x, rho[y, x], exact)


def test_moments_match_eq2():
    lx, ly = 33, 20
    f = noisy_state(lx, ly, 9)
    p = M.Params(lx, ly, tau=0.8)
    lat = make(p)
    got = [t.cpu().numpy() for t in lat.moments(to_dev(f))]
    ref = M.moments(M.physical(f))
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-13 * np.abs(r).max() + 1e-16


def test_fp32_shifted_one_step_and_moments():
    lx, ly = 64, 40
    rho0 = 1.1
    p = M.Params(lx, ly, tau=0.7, g=1e-3, t_top=0.8, t_bottom=1.2)
    f = noisy_state(lx, ly, 300, eps=0.02)
    d = encode32(f, rho0)
    fin = decode32(d, rho0)          # the exact input the fp32 path sees
    want = M.step(fin, p)
    lat = make(p, precision="fp32", rho0=rho0)
    lat.set_state(to_dev(d, torch.float32))
    lat.step(1)
    got = decode32(lat.state().cpu().numpy(), rho0)
    assert plane_err(got, want) <= 2e-6
    fields = [t.cpu().numpy() for t in lat.moments()]
    ref = M.moments(M.physical(decode32(encode32(want, rho0), rho0)))
    for g, r in zip(fields, ref):
        assert np.abs(g - r).max() <= 1e-6 * np.abs(r).max() + 1e-9


def test_fp32_propagate_bc_moves_bits():
    # Slots away from the walls are pure moves of the stored float32 bits.
    lx, ly = 40, 20
    p = M.Params(lx, ly, tau=0.7, t_top=0.8, t_bottom=1.2)
    d = encode32(noisy_state(lx, ly, 301), 1.0)
    lat = make(p, precision="fp32", rho0=1.0)
    got = lat.propagate_bc(to_dev(d, torch.float32)).cpu().numpy()
    want = M.propagate(d.astype(np.float64), p).astype(np.float32)
    np.testing.assert_array_equal(M.physical(got)[:, 3:ly - 3], M.physical(want)[:, 3:ly - 3])


def test_check_finite_and_status():
    p = M.Params(16, 12, tau=0.8)
    lat = make(p)
    f = noisy_state(16, 12, 5)
    lat.set_state(to_dev(f))
    assert lat.check_finite()
    f[4, 7, 3] = np.inf
    lat.set_state(to_dev(f))
    assert not lat.check_finite()
    assert lat.status() == 0


def _fields_err(a, b):
    return [np.abs(x - y).max() / np.abs(y).max() for x, y in zip(a, b)]


def test_fp32_shifted_error_stays_flat_over_1000_steps():
    # 64 x 128 RT lattice, stable contrast T = 0.75 / 1.25, tau = 0.6: the
    # float32 path against the float64 path (pinned to the oracle above).
    # A conservation leak in the float32 collide grows the rho / T error
    # linearly with the step count; storage rounding alone keeps it flat.
    rho, ux, uy, T, tt, tb = synth.rt_fields(64, 128, 4, 0, delta=0.5)
    kw = dict(tau=0.6, g=1e-5, t_top=tt, t_bottom=tb)
    a = Lattice(64, 128, precision="fp64", **kw).init(rho, ux, uy, T)
    b = Lattice(64, 128, precision="fp32", rho0=float(rho.mean()), **kw).init(rho, ux, uy, T)
    errs = {}
    for n in (200, 800):
        a.step(n)
        b.step(n)
        ea = [t.cpu().numpy() for t in a.moments()]
        eb = [t.cpu().numpy() for t in b.moments()]
        errs[n] = _fields_err(eb, ea)
    for n in (200, 800):
        assert errs[n][0] <= 1e-6 and errs[n][3] <= 1e-6, errs
    # no linear growth: 5x the steps, far less than 5x the error
    assert errs[800][0] <= 2.5 * errs[200][0] + 1e-7 and errs[800][3] <= 2.5 * errs[200][3] + 1e-7, errs


def test_fp32_shifted_conserves_mass():
    lx, ly = 48, 40
    rho, ux, uy, T = synth.random_fields(lx, ly, 77, umax=0.05, rho_range=(0.9, 1.1), t_range=(0.9, 1.1))
    lat = Lattice(lx, ly, tau=0.7, g=0.0, precision="fp32", rho0=1.0, periodic_y=True)
    lat.init(rho, ux, uy, T)
    m0 = lat.moments()[0].sum().item()
    lat.step(500)
    m1 = lat.moments()[0].sum().item()
    assert abs(m1 - m0) <= 1e-9 * m0, (m0, m1)


# ---------------------------------------------------------------------------
# float64 storage with the collide in double-float arithmetic (LBM_FP64_DF):
# held to the same bar as the float64 path.

@pytest.mark.parametrize("lx,ly", [(64, 128), (67, 45), (3, 6)])
@pytest.mark.parametrize("periodic_y", [False, True])
def test_one_step_parity_fp64df(lx, ly, periodic_y):
    p = M.Params(lx, ly, tau=0.7, g=2e-3, t_top=0.8, t_bottom=1.2, periodic_y=periodic_y)
    f = noisy_state(lx, ly, 200 + lx, eps=0.05)
    want = M.step(f, p)
    lat = make(p, precision="fp64df")
    lat.set_state(to_dev(f))
    lat.step(1)
    got = lat.state().cpu().numpy()
    assert np.isnan(got[:, :3]).all() and np.isnan(got[:, -3:]).all()
    assert plane_err(got, want) <= 1e-12


def test_rayleigh_taylor_64x128_100_steps_fp64df():
    rho, ux, uy, T, tt, tb = synth.rt_fields(64, 128, 4, 0)
    p = M.Params(64, 128, tau=0.8, g=1e-4, t_top=tt, t_bottom=tb)
    f0 = M.init_state(rho, ux, uy, T)
    lat = make(p, precision="fp64df")
    lat.set_state(to_dev(f0))
    lat.step(100)
    want = M.run(f0, p, 100)
    assert plane_err(lat.state().cpu().numpy(), want) <= 1e-12


# ---------------------------------------------------------------------------
# Regularised collide (LBM_FLAG_REGULARIZED): the oracle projects with explicit
# tensor Hermite polynomials; the kernel with velocity monomials and an inverse
# Gram matrix.  Same float64 bar.

@pytest.mark.parametrize("lx,ly", [(40, 24), (67, 45), (3, 6)])
@pytest.mark.parametrize("periodic_y", [False, True])
def test_one_step_parity_regularized(lx, ly, periodic_y):
    p = M.Params(lx, ly, tau=0.7, g=2e-3, t_top=0.8, t_bottom=1.2, periodic_y=periodic_y)
    f = noisy_state(lx, ly, 400 + lx, eps=0.05)
    want = M.step_regularized(f, p)
    lat = Lattice(lx, ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom, periodic_y=periodic_y,
                  regularized=True)
    lat.set_state(to_dev(f))
    lat.step(1)
    assert plane_err(lat.state().cpu().numpy(), want) <= 1e-12


def test_one_step_parity_bgk_outside_the_fixed_point_range():
    # The float64 BGK collide evaluates the equilibrium polynomial in fixed
    # point; a site whose equilibrium coefficients leave their degree-graded
    # range (a very hot or very fast site) relaxes in float64 instead, and a
    # population >= 4 sends the moment sums to float64.  All paths match the
    # oracle.
    lx, ly = 37, 11
    p = M.Params(lx, ly, tau=0.7, g=1e-3, t_top=0.9, t_bottom=1.1)
    rho, ux, uy, T = synth.random_fields(lx, ly, 433, umax=0.08)
    T[2, 7] = 60.0                                         # theta^2 terms beyond 2^10
    ux[6, 12] = 3.0                                        # degree-4 velocity terms beyond 2^2
    rho[4, 25] = 30.0                                      # populations >= 4, coefficients in range
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] *= 1.0 + 0.02 * synth.noise(lx, ly, 434)
    phys = f[:, 3:-3]
    phys[21, 1, 3] = 0.0
    phys[30, 8, 33] = 1e-300
    want = M.physical(M.step(f, p))
    lat = make(p)
    lat.set_state(to_dev(f))
    lat.step(1)
    got = M.physical(lat.state().cpu().numpy())
    # per site: the hot site's populations (~500) would hide errors elsewhere
    # in a per-plane scale
    site_err = np.abs(got - want).max(axis=0) / np.abs(want).max(axis=0)
    assert site_err.max() <= 1e-12


def test_one_step_parity_regularized_outside_the_fixed_point_range():
    # Sites whose pulled populations include one >= 4 (or whose projection
    # coefficients leave the fixed-point range) relax in float64; tiny, zero
    # and negative populations stay on the fixed-point path.  Both must match.
    lx, ly = 37, 11
    p = M.Params(lx, ly, tau=0.7, g=1e-3, t_top=0.9, t_bottom=1.1)
    f = noisy_state(lx, ly, 431, eps=0.05)
    phys = f[:, 3:-3]
    phys[9, 5, 20] = 4.5
    phys[0, 2, 7] = 6.0
    phys[21, 8, 30] = -0.01
    phys[11, 1, 3] = 0.0
    phys[30, 6, 33] = 1e-300
    want = M.step_regularized(f, p)
    lat = Lattice(lx, ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom, regularized=True)
    lat.set_state(to_dev(f))
    lat.step(1)
    assert plane_err(lat.state().cpu().numpy(), want) <= 1e-12


def test_rayleigh_taylor_64x128_100_steps_regularized():
    rho, ux, uy, T, tt, tb = synth.rt_fields(64, 128, 4, 0)
    p = M.Params(64, 128, tau=0.8, g=1e-4, t_top=tt, t_bottom=tb)
    f = M.init_state(rho, ux, uy, T)
    lat = Lattice(64, 128, tau=p.tau, g=p.g, t_top=tt, t_bottom=tb, regularized=True)
    lat.set_state(to_dev(f))
    lat.step(100)
    for _ in range(100):
        f = M.step_regularized(f, p)
    assert plane_err(lat.state().cpu().numpy(), f) <= 1e-12


def test_adjoint_refuses_regularized_context():
    from paper_1703_00186_gb300._lib import LBMError
    lat = Lattice(16, 12, tau=0.8, regularized=True)
    f = lat.new_state(0.1)
    with pytest.raises(LBMError):
        lat.adjoint_step(f, lat.new_cotangent(0.0))


# ---------------------------------------------------------------------------
# Degenerate cases

@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp64df"])
def test_uniform_periodic_state_stays_uniform_on_gpu(precision):
    lx, ly = 40, 20
    z = np.zeros((ly, lx))
    lat = Lattice(lx, ly, tau=0.7, g=1e-3, precision=precision, rho0=1.2, periodic_y=True)
    lat.init(z + 1.3, z + 0.05, z - 0.02, z + 0.9).step(5)
    s = lat.state().cpu().numpy()[:, 3:-3]
    for l in range(37):
        assert np.all(s[l] == s[l, 0, 0]), l


def rest_rounding_bound(T, tau, steps, unit):
    # At rest the equilibrium over w rho is, in powers of c2 = |c_l|^2 (the
    # monomial form the step evaluates, theta = T - 1),
    #   P = (1 - theta + theta^2) + theta (1/2 - theta) c2 + theta^2 c2^2 / 8.
    # The step's float64 equilibrium and the state's (rounded by the oracle)
    # each carry a few roundings of these terms, so they differ relatively by
    # about kappa units, kappa = sum |terms| / |P| (8.9 on the outer shells
    # at T = 0.85); the relaxation moves f by omega times that per step, and
    # the moments the next step reads have moved by as much.
    th, c2 = T - 1.0, K["c2"]
    terms = np.array([np.full_like(c2, 1 - th + th * th), th * (0.5 - th) * c2, th * th * c2 * c2 / 8])
    kappa = (np.abs(terms).sum(axis=0) / np.abs(terms.sum(axis=0))).max()
    return steps * (1.0 / tau) * kappa * 4 * unit


@pytest.mark.parametrize("precision", ["fp64", "fp64df"])
def test_rest_equilibrium_is_a_fixed_point_of_the_step_on_gpu(precision):
    # a uniform fluid at rest without gravity is a fixed point of
    # propagate + collide (periodic in y: no walls); 3 steps move it by
    # rounding only.  float64: unit 2^-53 (measured 1.1e-14 against a bound
    # of 2.0e-14); double-float collide: its equilibrium sums are accurate to
    # ~2^-46, bound 1e-13
    lx, ly, T, tau, steps = 33, 17, 0.85, 0.6, 3
    z = np.zeros((ly, lx))
    f = M.init_state(z + 1.25, z, z, z + T)
    lat = make(M.Params(lx, ly, tau=tau, g=0.0, periodic_y=True), precision=precision)
    lat.set_state(to_dev(f))
    lat.step(steps)
    tol = rest_rounding_bound(T, tau, steps, 2.0 ** -53) if precision == "fp64" else 1e-13
    assert plane_err(lat.state().cpu().numpy(), f) <= tol


def test_zero_steps_is_a_no_op():
    p = M.Params(16, 12, tau=0.8)
    lat = make(p)
    f = noisy_state(16, 12, 9)
    lat.set_state(to_dev(f))
    lat.step(0)
    np.testing.assert_array_equal(M.physical(lat.state().cpu().numpy()), M.physical(f))


def test_state_larger_than_2_to_31_elements_uses_64_bit_indexing():
    # 16384 x 4096 float32: 37 * 4102 * 16384 = 2.49e9 elements per state.
    lx, ly = 16384, 4096
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 8, 3, delta=0.5)
    rho0 = float(rho.mean())
    lat = Lattice(lx, ly, tau=0.7, g=1e-4, t_top=tt, t_bottom=tb, precision="fp32", rho0=rho0)
    assert 37 * (ly + 6) * lx > 2 ** 31
    lat.init(rho, ux, uy, T).step(1)
    p = M.Params(lx, ly, tau=0.7, g=1e-4, t_top=tt, t_bottom=tb)
    state = lat.state()
    for x0 in (0, lx - 8):   # the last columns of the top rows sit past 2^31
        pad = 6
        cols = (x0 - pad + np.arange(8 + 2 * pad)) % lx
        q = M.Params(len(cols), ly, tau=p.tau, g=p.g, t_top=tt, t_bottom=tb)
        f = M.init_state(*[np.ascontiguousarray(a[:, cols]) for a in (rho, ux, uy, T)])
        f[:, 3:-3] = decode32(encode32(f, rho0), rho0)[:, 3:-3]
        want = M.physical(M.step(f, q))[:, :, pad:pad + 8]
        got = decode32(state[:, 3:-3, x0:x0 + 8].cpu().numpy(), rho0)
        scale = np.abs(want).max(axis=(1, 2))
        assert (np.abs(got - want).max(axis=(1, 2)) / scale).max() <= 2e-6, x0


# ---------------------------------------------------------------------------
# Boundary paths: checkpoint through pinned host memory, explicit-buffer step

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_round_trip_through_pinned_host_memory(precision):
    lx, ly = 50, 22
    rho, ux, uy, T = synth.random_fields(lx, ly, 11)
    lat = Lattice(lx, ly, tau=0.7, g=1e-3, t_top=0.9, t_bottom=1.1, precision=precision, rho0=1.1)
    lat.init(rho, ux, uy, T).step(3)
    host = torch.empty(lat.shape, dtype=lat.dtype, pin_memory=True)
    lat.get_state(host)
    torch.cuda.synchronize()
    ref = lat.state().clone()
    lat.step(4)                       # move on, then restore the checkpoint
    lat.set_state(host)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(lat.state()[:, 3:-3].cpu().numpy(), ref[:, 3:-3].cpu().numpy())
    lat.step(4)
    again = lat.state().clone()
    lat.set_state(host).step(4)
    np.testing.assert_array_equal(lat.state()[:, 3:-3].cpu().numpy(), again[:, 3:-3].cpu().numpy())


def test_step_from_equals_step():
    lx, ly = 41, 19
    rho, ux, uy, T = synth.random_fields(lx, ly, 12)
    lat = Lattice(lx, ly, tau=0.7, g=1e-3, t_top=0.9, t_bottom=1.1).init(rho, ux, uy, T)
    src = lat.state().clone()
    dst = lat.new_state()
    lat.step_from(src, dst)
    lat.step(1)
    np.testing.assert_array_equal(dst[:, 3:-3].cpu().numpy(), lat.state()[:, 3:-3].cpu().numpy())


def test_host_or_mistyped_tensors_are_refused_before_any_launch():
    # The binding checks every tensor it hands to a kernel; nothing reaches
    # the device, and the lattice steps normally afterwards.
    lat = Lattice(16, 12, tau=0.8)
    host = torch.zeros(lat.shape, dtype=torch.float64)
    dev = lat.new_state(0.1)
    with pytest.raises(ValueError):
        lat.step_from(host, lat.new_state())
    with pytest.raises(ValueError):
        lat.propagate_bc(host)
    with pytest.raises(ValueError):
        lat.adjoint_step(dev, host)
    with pytest.raises(ValueError):
        lat.adjoint_step(dev.float(), lat.new_cotangent(0.0))
    with pytest.raises(ValueError):
        lat.moments(host)
    with pytest.raises(ValueError):
        lat.check_finite(dev[:, :, :8])
    rho, ux, uy, T = synth.random_fields(16, 12, 5)
    lat.init(rho, ux, uy, T).step(2)
    assert lat.status() == 0 and lat.check_finite()


# ---------------------------------------------------------------------------
# FP32 shifted storage: the TMA-staged step against the plain-load step.

@pytest.mark.parametrize("lx,ly", [(64, 40), (100, 37), (36, 6), (8, 9), (2048, 64)])
def test_fp32_tma_staged_step_is_bit_identical_to_plain_loads(lx, ly):
    # ragged tiles in x (100, 36, 8) and y (37, 9), seam columns read with
    # plain loads, wall rows, and a row of many tiles
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 2, 5, delta=0.4)
    kw = dict(tau=0.7, g=1e-4, t_top=tt, t_bottom=tb, precision="fp32", rho0=float(rho.mean()))
    a = Lattice(lx, ly, tma_loads=True, **kw).init(rho, ux, uy, T)
    b = Lattice(lx, ly, **kw).init(rho, ux, uy, T)
    assert a.step_path() == "tma" and b.step_path() == "plain"
    a.step(7)
    b.step(7)
    assert a.status() == 0 and b.status() == 0
    assert torch.equal(a.state()[:, 3:-3], b.state()[:, 3:-3])


def test_fp32_step_path_falls_back_to_plain_loads():
    kw = dict(tau=0.7, precision="fp32", tma_loads=True)
    assert Lattice(66, 12, **kw).step_path() == "plain"                    # lx not a multiple of 4
    assert Lattice(64, 12, periodic_y=True, **kw).step_path() == "plain"   # y wraps
    assert Lattice(64, 12, tau=0.7, tma_loads=True).step_path() == "plain"  # float64 modes
    assert Lattice(64, 12, tau=0.7, precision="fp32").step_path() == "plain"  # not requested


@pytest.mark.parametrize("precision", ["fp64", "fp64df"])
def test_non_finite_population_stays_local_and_non_finite(precision):
    # An infinite population makes its site's moments non-finite (NaN); after
    # one step exactly the sites that pull from it, or from the same column
    # sums, are non-finite, as in the oracle, and every other site still
    # matches the oracle.
    lx, ly = 24, 20
    p = M.Params(lx, ly, tau=0.7, g=1e-3, t_top=0.9, t_bottom=1.1)
    f = noisy_state(lx, ly, 95)
    f[7, 3 + 10, 12] = np.inf
    with np.errstate(invalid="ignore", over="ignore"):
        want = M.step(f, p)
    lat = make(p, precision=precision)
    lat.set_state(to_dev(f))
    lat.step(1)
    got = lat.state().cpu().numpy()
    gw, ww = M.physical(got), M.physical(want)
    fin = np.isfinite(ww).all(axis=0)
    assert (~fin).any()
    np.testing.assert_array_equal(np.isfinite(gw).all(axis=0), fin)
    scale = np.abs(ww[:, fin]).max(axis=1)
    assert (np.abs(gw[:, fin] - ww[:, fin]).max(axis=1) / scale).max() <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_step_equals_plain_step(precision):
    # lbm_step_graph replays the same launches from a cached CUDA graph: bit
    # for bit the plain steps, for odd and even n and for repeated calls
    rho, ux, uy, T, tt, tb = synth.rt_fields(64, 128, 4, 0)
    kw = dict(tau=0.8, g=1e-4, t_top=tt, t_bottom=tb, precision=precision, rho0=float(rho.mean()))
    a = Lattice(64, 128, **kw).init(rho, ux, uy, T)
    b = Lattice(64, 128, **kw).init(rho, ux, uy, T)
    for n in (3, 3, 4, 0, 7):
        a.step(n)
        b.step(n, graph=True)
    assert torch.equal(M.physical(a.state()), M.physical(b.state()))
    assert b.status() == 0
