"""Pins of the oracle's D2Q37 step against what the model fixes (CPU only).

Each test checks a fact independent of the oracle's own formulas: Maxwellian
moments, conservation laws, the exact effect of the gravity shift, the
direction of streaming, mass balance at the walls, permutation structure.
"""
import math

import numpy as np
import pytest

import synth
from oracle import lattice, model as M

K = lattice.constants()


def gauss_moment_1d(u, T, k):
    """E[(u + sqrt(T) z)^k] for a unit normal z (binomial expansion)."""
    out = 0.0
    for j in range(0, k + 1, 2):
        out = out + math.comb(k, j) * u ** (k - j) * T ** (j // 2) * math.prod(range(j - 1, 0, -2))
    return out


def rand_fields(n, seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, n)
    ux = rng.uniform(-0.2, 0.2, n)
    uy = rng.uniform(-0.2, 0.2, n)
    T = rng.uniform(0.6, 1.4, n)
    return rho, ux, uy, T


def test_equilibrium_moments_are_maxwellian_to_order_4():
    rho, ux, uy, T = rand_fields(50, 1)
    feq = M.equilibrium(rho, ux, uy, T)
    c = K["c"]
    for a in range(5):
        for b in range(5 - a):
            got = np.tensordot(c[:, 0] ** a * c[:, 1] ** b, feq, axes=(0, 0))
            want = rho * gauss_moment_1d(ux, T, a) * gauss_moment_1d(uy, T, b)
            np.testing.assert_allclose(got, want, rtol=2e-13, atol=2e-14)


def test_equilibrium_order5_moment_is_not_maxwellian():
    # A 4th-order expansion cannot reproduce 5th-order moments when u != 0.
    rho, ux, uy, T = np.array([1.0]), np.array([0.2]), np.array([0.1]), np.array([1.2])
    feq = M.equilibrium(rho, ux, uy, T)
    got = float(np.tensordot(K["c"][:, 0] ** 5, feq, axes=(0, 0))[0])
    want = float(gauss_moment_1d(ux, T, 5)[0])
    assert abs(got - want) > 1e-6


def test_equilibrium_closed_form_equals_hermite_tensor_sum():
    rho, ux, uy, T = rand_fields(40, 2)
    a = M.equilibrium(rho, ux, uy, T)
    b = M.equilibrium_hermite(rho, ux, uy, T)
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-16)


def test_equilibrium_at_rest_and_unit_temperature_is_weights():
    feq = M.equilibrium(np.array(1.7), np.array(0.0), np.array(0.0), np.array(1.0))
    np.testing.assert_array_equal(feq, K["w"] * 1.7)


def test_moments_recover_fields():
    rho, ux, uy, T = rand_fields(30, 3)
    r2, ux2, uy2, T2 = M.moments(M.equilibrium(rho, ux, uy, T))
    np.testing.assert_allclose(r2, rho, rtol=1e-14)
    np.testing.assert_allclose(ux2, ux, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(uy2, uy, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(T2, T, rtol=1e-13)


def _noisy_state(lx, ly, seed, eps=0.02):
    rho, ux, uy, T = synth.random_fields(lx, ly, seed)
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] *= 1.0 + eps * synth.noise(lx, ly, seed + 1)
    return f


def _conserved(fp):
    c = K["c"]
    rho = fp.sum(0)
    jx = np.tensordot(c[:, 0], fp, axes=(0, 0))
    jy = np.tensordot(c[:, 1], fp, axes=(0, 0))
    e = np.tensordot(c[:, 0] ** 2 + c[:, 1] ** 2, fp, axes=(0, 0))
    return rho, jx, jy, e


def test_collide_conserves_mass_momentum_energy_without_gravity():
    f = _noisy_state(8, 6, 10)
    p = M.Params(8, 6, tau=0.7, g=0.0)
    out = M.collide(f, p)
    for a, b in zip(_conserved(M.physical(f)), _conserved(M.physical(out))):
        np.testing.assert_allclose(b, a, rtol=1e-13, atol=1e-14)
    assert np.abs(M.physical(out) - M.physical(f)).max() > 1e-4  # it did relax


def test_collide_gravity_adds_rho_g_and_keeps_rho_and_T():
    f = _noisy_state(8, 6, 11)
    g = 3e-3
    p = M.Params(8, 6, tau=0.65, g=g)
    out = M.collide(f, p)
    r0, jx0, jy0, _ = _conserved(M.physical(f))
    r1, jx1, jy1, _ = _conserved(M.physical(out))
    np.testing.assert_allclose(r1, r0, rtol=1e-14)
    np.testing.assert_allclose(jx1, jx0, atol=1e-14)
    np.testing.assert_allclose(jy1, jy0 - r0 * g, rtol=1e-12, atol=1e-14)
    T0 = M.moments(M.physical(f))[3]
    T1 = M.moments(M.physical(out))[3]
    np.testing.assert_allclose(T1, T0, rtol=1e-13)


def test_equilibrium_is_fixed_point_of_collide():
    rho, ux, uy, T = synth.random_fields(6, 7, 12)
    f = M.init_state(rho, ux, uy, T)
    out = M.collide(f, M.Params(6, 7, tau=0.6, g=0.0))
    np.testing.assert_allclose(M.physical(out), M.physical(f), rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("periodic_y", [False, True])
def test_propagate_moves_population_along_its_velocity(periodic_y):
    lx, ly = 11, 13
    p = M.Params(lx, ly, tau=1.0, periodic_y=periodic_y)
    x0, y0 = 4, 6
    for l in range(37):
        f = np.zeros((37, ly + 6, lx))
        f[l, 3 + y0, x0] = 1.0
        out = M.propagate(f, p)
        ax, ay = K["xi"][l]
        tgt = np.zeros((ly, lx))
        tgt[y0 + ay, (x0 + ax) % lx] = 1.0
        np.testing.assert_array_equal(M.physical(out)[l], tgt)


def test_propagate_wraps_periodically_in_x():
    lx, ly = 5, 9
    p = M.Params(lx, ly, tau=1.0)
    f = np.zeros((37, ly + 6, lx))
    l = int(np.where((K["xi"] == [3, 1]).all(1))[0][0])
    f[l, 3 + 4, 4] = 1.0
    out = M.propagate(f, p)
    assert M.physical(out)[l, 5, (4 + 3) % lx] == 1.0


def test_periodic_propagate_is_a_permutation_undone_by_reverse_shift():
    lx, ly = 9, 10
    p = M.Params(lx, ly, tau=1.0, periodic_y=True)
    rng = np.random.default_rng(5)
    f = np.full((37, ly + 6, lx), np.nan)
    f[:, 3:-3] = rng.standard_normal((37, ly, lx))
    out = M.propagate(f, p)
    for l in range(37):
        np.testing.assert_array_equal(np.sort(M.physical(out)[l].ravel()),
                                      np.sort(M.physical(f)[l].ravel()))
        ax, ay = K["xi"][l]
        back = np.roll(np.roll(M.physical(out)[l], -ay, axis=0), -ax, axis=1)
        np.testing.assert_array_equal(back, M.physical(f)[l])


def test_walls_conserve_mass_exactly_and_ignore_halos():
    lx, ly = 10, 12
    f = _noisy_state(lx, ly, 20, eps=0.2)
    f[:, :3] = np.nan
    f[:, -3:] = np.nan
    p = M.Params(lx, ly, tau=0.9, t_top=0.7, t_bottom=1.3)
    out = M.propagate_bc(f, p)
    assert np.isfinite(M.physical(out)).all()
    m0 = M.physical(f).sum()
    m1 = M.physical(out).sum()
    assert abs(m1 - m0) <= 1e-14 * m0
    # and per column: what left through the walls landing in column x returns there
    pure = M.propagate(np.nan_to_num(f, nan=0.0), p)
    lost = M.physical(np.nan_to_num(f, nan=0.0)).sum() - M.physical(pure).sum()
    assert lost > 0


def test_wall_unknown_slots_follow_wall_equilibrium_ratios():
    lx, ly = 7, 10
    f = _noisy_state(lx, ly, 21, eps=0.3)
    p = M.Params(lx, ly, tau=0.9, t_top=0.8, t_bottom=1.25)
    out = M.physical(M.propagate_bc(f, p))
    for wall, Tw in (("bottom", 1.25), ("top", 0.8)):
        phi = M.equilibrium(np.array(1.0), np.array(0.0), np.array(0.0), np.array(Tw))
        slots = M.unknown_slots(wall)
        assert len(slots) == 26
        d0, l0 = slots[0]
        y0 = d0 if wall == "bottom" else ly - 1 - d0
        for (d, l) in slots:
            y = d if wall == "bottom" else ly - 1 - d
            np.testing.assert_allclose(out[l, y] / out[l0, y0], phi[l] / phi[l0], rtol=1e-13)


def test_wall_q_at_unit_temperature_is_weight_ratio():
    # phi = w at T = 1, so q_l = w_l / sum over the 26 slots of w.
    for wall in ("bottom", "top"):
        q = M.wall_q(1.0, wall)
        slots = M.unknown_slots(wall)
        tot = sum(K["w"][l] for (_, l) in slots)
        for (_, l) in slots:
            assert q[l] == pytest.approx(K["w"][l] / tot, rel=1e-15)
    assert sorted(M.wall_q(1.3, "bottom")[M.wall_q(1.3, "bottom") > 0]) == \
        sorted(M.wall_q(1.3, "top")[M.wall_q(1.3, "top") > 0])


def test_rows_away_from_walls_are_pure_propagate():
    lx, ly = 8, 14
    f = _noisy_state(lx, ly, 22)
    p = M.Params(lx, ly, tau=0.9, t_top=0.9, t_bottom=1.1)
    pure = M.physical(M.propagate(f, p))
    out = M.physical(M.propagate_bc(f, p))
    np.testing.assert_array_equal(out[:, 3:ly - 3], pure[:, 3:ly - 3])
    # near the walls, every slot whose source is physical is also pure propagate
    for y in list(range(3)) + list(range(ly - 3, ly)):
        for l in range(37):
            if 0 <= y - K["xi"][l, 1] < ly:
                np.testing.assert_array_equal(out[l, y], pure[l, y])


def test_uniform_periodic_state_stays_uniform():
    lx, ly = 6, 8
    f = M.init_state(np.full((ly, lx), 1.3), np.full((ly, lx), 0.05),
                     np.full((ly, lx), -0.02), np.full((ly, lx), 0.9))
    p = M.Params(lx, ly, tau=0.7, g=1e-3, periodic_y=True)
    for _ in range(4):
        f = M.step(f, p)
    fp = M.physical(f)
    for l in range(37):
        assert np.all(fp[l] == fp[l, 0, 0])
    # gravity accelerated the uniform fluid by exactly g per step
    _, _, uy, _ = M.moments(fp)
    assert uy[0, 0] == pytest.approx(-0.02 - 4e-3, rel=1e-12)


def test_walled_lattice_conserves_total_mass_over_steps():
    rho, ux, uy, T, tt, tb = synth.rt_fields(16, 20, 3, 7)
    p = M.Params(16, 20, tau=0.8, g=1e-3, t_top=tt, t_bottom=tb)
    f = M.init_state(rho, ux, uy, T)
    m0 = M.physical(f).sum()
    f = M.run(f, p, 10)
    assert abs(M.physical(f).sum() - m0) <= 1e-13 * m0
