"""Pins of the oracle's regularised (Hermite-projected) collide (CPU only).

The projection is pinned by facts independent of its code: it keeps every
moment of order <= 4 (checked against direct sums), it is idempotent, it
leaves an order-4 polynomial times w unchanged (the equilibrium), and it
removes a degree-5 Hermite polynomial times w, which is orthogonal to the
order-<=4 space under the order-9 quadrature.
"""
import itertools

import numpy as np

import synth
from oracle import lattice, model as M

K = lattice.constants()


def monomial_moments(fp, deg=4):
    c = K["c"]
    out = {}
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            out[(a, b)] = np.tensordot(c[:, 0] ** a * c[:, 1] ** b, fp, axes=(0, 0))
    return out


def rand_pop(shape, seed):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(37,) + shape)


def test_projection_keeps_moments_to_order_4():
    f = rand_pop((3, 4), 1)
    pf = M.hermite_project(f)
    mf, mp = monomial_moments(f), monomial_moments(pf)
    for key in mf:
        np.testing.assert_allclose(mp[key], mf[key], rtol=1e-12, atol=1e-13)


def test_projection_is_idempotent_and_keeps_equilibrium():
    f = rand_pop((5,), 2)
    pf = M.hermite_project(f)
    np.testing.assert_allclose(M.hermite_project(pf), pf, rtol=1e-12, atol=1e-14)
    rho, ux, uy, T = synth.random_fields(4, 3, 3)
    feq = M.equilibrium(rho, ux, uy, T)
    np.testing.assert_allclose(M.hermite_project(feq), feq, rtol=1e-12, atol=1e-15)


def test_projection_removes_a_fifth_order_hermite_mode():
    # w_l He5(c_lx) with He5(x) = x^5 - 10 x^3 + 15 x (probabilists' Hermite)
    cx = K["c"][:, 0]
    ghost = K["w"] * (cx ** 5 - 10 * cx ** 3 + 15 * cx)
    assert np.abs(ghost).max() > 1e-3
    np.testing.assert_allclose(M.hermite_project(ghost[:, None]), 0.0, atol=1e-14)


def test_projection_space_has_dimension_15():
    basis = np.eye(37)
    proj = M.hermite_project(basis)          # (37, 37): column j = Pi e_j
    assert np.linalg.matrix_rank(proj, tol=1e-10) == 15


def test_regularized_collide_conserves_like_bgk():
    lx, ly = 6, 7
    rho, ux, uy, T = synth.random_fields(lx, ly, 4)
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] *= 1.0 + 0.05 * synth.noise(lx, ly, 5)
    p = M.Params(lx, ly, tau=0.7, g=2e-3)
    a = M.collide(f, p)
    b = M.collide_regularized(f, p)
    for (key, ma), mb in zip(monomial_moments(M.physical(a), 2).items(),
                             monomial_moments(M.physical(b), 2).values()):
        if key[0] + key[1] <= 1 or key in ((2, 0), (0, 2)):
            # mass, momentum and the energy trace agree with plain BGK
            np.testing.assert_allclose(mb, ma, rtol=1e-12, atol=1e-14)
    # the two differ: the regularised collide removes the ghost components
    assert np.abs(M.physical(a) - M.physical(b)).max() > 1e-6


def test_regularized_equals_bgk_inside_the_hermite_space():
    lx, ly = 5, 6
    rho, ux, uy, T = synth.random_fields(lx, ly, 6)
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] = M.hermite_project(f[:, 3:-3] * (1.0 + 0.05 * synth.noise(lx, ly, 7)))
    p = M.Params(lx, ly, tau=0.65, g=1e-3)
    np.testing.assert_allclose(M.physical(M.collide_regularized(f, p)), M.physical(M.collide(f, p)),
                               rtol=1e-12, atol=1e-15)
