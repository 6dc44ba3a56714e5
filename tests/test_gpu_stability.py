"""The GPU step is unstable exactly where the oracle's linear analysis says.

``oracle.stability`` gives the largest growth factor per step of a
perturbation of a uniform fluid at rest (the complex-step Jacobian of the
oracle's collide times the propagate shift symbol).  On a 16 x 16 periodic
lattice at T = 0.5, tau = 0.6 (the cold layer of the stated Rayleigh-Taylor
workload) a 1e-8 perturbation stepped by the float64 kernel grows at that
factor, maximised over the lattice's own wavevectors, within 1e-3; at
T = 0.75 it decays.  This is the mechanism by which the stated 2048 x 4096
workload loses finiteness after about 200 steps.
"""
import numpy as np
import pytest

from oracle import model as M, stability as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1703_00186_gb300.lbm import Lattice

N = 16


def _amplitudes(T, steps, marks):
    f = M.init_state(np.ones((N, N)), np.zeros((N, N)), np.zeros((N, N)), np.full((N, N), T))
    f[:, 3:-3] *= 1.0 + 1e-8 * np.random.default_rng(0).uniform(-1.0, 1.0, size=(M.NPOP, N, N))
    lat = Lattice(N, N, tau=0.6, g=0.0, periodic_y=True)
    lat.set_state(torch.as_tensor(f, device="cuda"))
    out, done = {}, 0
    for m in marks:
        lat.step(m - done)
        done = m
        ph = M.physical(lat.state().cpu().numpy())
        out[m] = np.abs(ph - ph.mean(axis=(1, 2), keepdims=True)).max()
    return out


def _lattice_radius(T, tau):
    J = S.collide_jacobian(T, tau)
    k = 2.0 * np.pi * np.arange(N) / N
    return max(np.abs(np.linalg.eigvals(J * S.shift_symbol(kx, ky)[None, :])).max() for kx in k for ky in k)


def test_gpu_growth_equals_the_oracle_linear_growth_factor():
    amp = _amplitudes(0.5, 200, (150, 200))
    rate = (amp[200] / amp[150]) ** (1.0 / 50.0)
    assert rate == pytest.approx(_lattice_radius(0.5, 0.6), rel=1e-3)


def test_gpu_perturbation_decays_at_the_stable_contrast():
    amp = _amplitudes(0.75, 100, (20, 100))
    assert amp[100] < amp[20] < 1e-8
