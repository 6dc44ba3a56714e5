"""Pins of the oracle's discrete adjoint (CPU only).

* dot-product tests: <A v, w> = <v, A^T w> with A v computed by the forward
  code (exactly, for the linear B P; by complex-step JVP for the full step);
* the rollout gradient against complex-step directional derivatives of the
  forward rollout and against float64 central finite differences.
"""
import numpy as np
import pytest

import synth
from oracle import adjoint as A, model as M


def inner(a, b):
    return float((M.physical(a) * M.physical(b)).sum())


def rand_state(lx, ly, seed):
    f = np.full((37, ly + 6, lx), np.nan)
    f[:, 3:-3] = np.random.default_rng(seed).standard_normal((37, ly, lx))
    return f


@pytest.mark.parametrize("periodic_y", [False, True])
def test_propagate_bc_transpose_dot_product(periodic_y):
    lx, ly = 9, 11
    p = M.Params(lx, ly, tau=0.8, t_top=0.7, t_bottom=1.3, periodic_y=periodic_y)
    v = rand_state(lx, ly, 1)
    w = rand_state(lx, ly, 2)
    lhs = inner(M.propagate_bc(v, p), w)
    rhs = inner(v, A.propagate_bc_transpose(w, p))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def _physical_state(lx, ly, seed):
    rho, ux, uy, T = synth.random_fields(lx, ly, seed, umax=0.08)
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] *= 1.0 + 0.03 * synth.noise(lx, ly, seed + 1)
    return f


def test_adjoint_step_dot_product_against_complex_step_jvp():
    lx, ly = 7, 10
    p = M.Params(lx, ly, tau=0.7, g=1e-3, t_top=0.9, t_bottom=1.15)
    f = _physical_state(lx, ly, 3)
    v = rand_state(lx, ly, 4)
    w = rand_state(lx, ly, 5)
    fc = f.astype(np.complex128) + 1j * A.H_CS * v
    jv = np.imag(M.step(fc, p)) / A.H_CS
    lhs = inner(jv, w)
    rhs = inner(v, A.adjoint_step(f, w, p))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


def test_moments_vjp_dot_product():
    lx, ly = 5, 7
    f = _physical_state(lx, ly, 6)
    v = rand_state(lx, ly, 7)
    rng = np.random.default_rng(8)
    g = [rng.standard_normal((ly, lx)) for _ in range(4)]
    fc = f.astype(np.complex128) + 1j * A.H_CS * v
    dm = [np.imag(x) / A.H_CS for x in M.moments(M.physical(fc))]
    lhs = sum(float((a * b).sum()) for a, b in zip(dm, g))
    rhs = inner(v, A.moments_vjp(f, *g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def _rollout_case():
    lx, ly = 8, 12
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 2, 9, delta=0.4, width=1.5)
    p = M.Params(lx, ly, tau=0.8, g=1e-3, t_top=tt, t_bottom=tb)
    target = T + synth.smooth_field(lx, ly, 10, amp=0.05)
    dT0 = 0.01 * synth.smooth_field(lx, ly, 11, amp=1.0)
    return p, rho, T, target, dT0


def test_rollout_gradient_matches_complex_step_directional_derivative():
    p, rho, T, target, dT0 = _rollout_case()
    n = 6
    grad = A.rollout_grad(dT0, rho, T, target, p, n)
    rng = np.random.default_rng(12)
    for _ in range(2):
        v = rng.standard_normal(dT0.shape)
        dd = np.imag(A.rollout_loss(dT0 + 1j * A.H_CS * v, rho, T, target, p, n)) / A.H_CS
        assert float((grad * v).sum()) == pytest.approx(dd, rel=1e-11)


def test_rollout_gradient_matches_central_finite_differences():
    p, rho, T, target, dT0 = _rollout_case()
    n = 6
    grad = A.rollout_grad(dT0, rho, T, target, p, n)
    v = np.random.default_rng(13).standard_normal(dT0.shape)
    eps = 1e-5
    jp = A.rollout_loss(dT0 + eps * v, rho, T, target, p, n)
    jm = A.rollout_loss(dT0 - eps * v, rho, T, target, p, n)
    fd = (jp - jm) / (2 * eps)
    assert float((grad * v).sum()) == pytest.approx(fd, rel=1e-6)
