"""Where the plain BGK D2Q37 step is stable (CPU): the stated Rayleigh-Taylor
contrast (cold layer T = 0.5, tau = 0.6) is linearly unstable, the stable
contrast of the error studies (T = 0.75 / 1.25) is not.

``oracle.stability`` linearises the oracle step about a uniform fluid at rest
(complex-step Jacobian of collide times the propagate shift symbol per
wavevector).  It is pinned here against the oracle's own time stepping: the
growth per step of a 1e-8 perturbation of a uniform periodic lattice equals
the largest spectral radius over that lattice's wavevectors, and a stable
state's perturbation decays.
"""
import numpy as np
import pytest

from oracle import lattice, model as M, stability as S

N = 16  # periodic lattice N x N


def _perturbed_uniform(T, seed=0):
    f = M.init_state(np.ones((N, N)), np.zeros((N, N)), np.zeros((N, N)), np.full((N, N), T))
    f[:, 3:-3] *= 1.0 + 1e-8 * np.random.default_rng(seed).uniform(-1.0, 1.0, size=(M.NPOP, N, N))
    return f


def _amplitude(f):
    ph = M.physical(f)
    return np.abs(ph - ph.mean(axis=(1, 2), keepdims=True)).max()


def _run(T, tau, steps, marks):
    p = M.Params(N, N, tau=tau, g=0.0, periodic_y=True)
    f = _perturbed_uniform(T)
    out = {}
    for i in range(1, steps + 1):
        f = M.step(f, p)
        if i in marks:
            out[i] = _amplitude(f)
    return out


def _lattice_radius(T, tau):
    J = S.collide_jacobian(T, tau)
    k = 2.0 * np.pi * np.arange(N) / N
    return max(np.abs(np.linalg.eigvals(J * S.shift_symbol(kx, ky)[None, :])).max() for kx in k for ky in k)


def test_time_domain_growth_equals_the_linear_growth_factor():
    amp = _run(0.5, 0.6, 200, (150, 200))
    rate = (amp[200] / amp[150]) ** (1.0 / 50.0)
    assert rate == pytest.approx(_lattice_radius(0.5, 0.6), rel=1e-3)
    assert amp[200] > 1e3 * 1e-8  # grew by orders of magnitude from 1e-8


def test_stable_contrast_perturbation_decays():
    amp = _run(0.75, 0.6, 100, (20, 100))
    assert amp[100] < amp[20] < 1e-8
    assert _lattice_radius(0.75, 0.6) <= 1.0 + 1e-12


def test_stated_cold_layer_is_unstable_the_error_study_contrast_is_not():
    r, kx, ky = S.max_growth(0.5, 0.6)
    assert r > 1.09  # e-folding in about 11 steps: roundoff reaches O(1) within a few hundred
    for T in (0.75, 1.25, 1.5):
        assert S.max_growth(T, 0.6)[0] <= 1.0 + 1e-12, T


def test_equilibrium_turns_negative_at_T05_on_the_xi2_5_shell():
    q, l = S.min_equilibrium_population(0.5)
    xi = lattice.constants()["xi"][l]
    assert q < 0.0 and int(xi @ xi) == 5
    for T in (0.6, 0.75, 1.25, 1.5):
        assert S.min_equilibrium_population(T)[0] > 0.0, T
