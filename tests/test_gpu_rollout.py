"""Checkpointed adjoint rollouts on the GPU (torch.autograd.Function).

* the gradient equals the oracle's discrete-adjoint gradient (float64 both
  sides; <= 1e-10 relative, the sweep accumulates rounding over the steps);
* it matches float64 central finite differences of the GPU forward rollout
  on 16 seeded directions to <= 1e-6 relative (the tolerance set for the
  adjoint);
* checkpoint spacing K does not change the result beyond rounding.
"""
import numpy as np
import pytest

import synth
from oracle import adjoint as A, model as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    from paper_1703_00186_gb300.adjoint import temperature_loss
    from paper_1703_00186_gb300.lbm import Lattice


def case(lx, ly, seed=3, delta=0.4):
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 3, seed, delta=delta, width=1.5)
    target = T + synth.smooth_field(lx, ly, seed + 1, amp=0.05)
    dT0 = 0.01 * synth.smooth_field(lx, ly, seed + 2, amp=1.0)
    p = M.Params(lx, ly, tau=0.8, g=1e-3, t_top=tt, t_bottom=tb)
    return p, rho, T, target, dT0


def gpu_grad(p, rho, T, target, dT0, n, K, precision="fp64"):
    lat = Lattice(p.lx, p.ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom,
                  precision=precision, rho0=float(rho.mean()))
    d = torch.tensor(dT0, device="cuda", requires_grad=True)
    J = temperature_loss(d, lat, torch.tensor(rho, device="cuda"), torch.tensor(T, device="cuda"),
                         torch.tensor(target, device="cuda"), n, K)
    J.backward()
    return float(J), d.grad.cpu().numpy(), lat


def test_rollout_gradient_matches_oracle_adjoint():
    p, rho, T, target, dT0 = case(12, 16)
    n = 9
    J, g, _ = gpu_grad(p, rho, T, target, dT0, n, K=4)
    Jo = A.rollout_loss(dT0, rho, T, target, p, n)
    go = A.rollout_grad(dT0, rho, T, target, p, n)
    assert J == pytest.approx(Jo, rel=1e-12)
    assert np.abs(g - go).max() <= 1e-10 * np.abs(go).max()


def test_checkpoint_spacing_does_not_change_gradient():
    p, rho, T, target, dT0 = case(32, 24)
    _, g1, _ = gpu_grad(p, rho, T, target, dT0, 30, K=30)
    _, g2, _ = gpu_grad(p, rho, T, target, dT0, 30, K=7)
    assert np.abs(g1 - g2).max() <= 1e-13 * np.abs(g1).max()


def _fp64_central_differences(p, rho, T, target, dT0, n, K, dirs, eps=1e-4):
    """float64 central differences of the float64 GPU rollout along dirs."""
    lat = Lattice(p.lx, p.ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom, precision="fp64")
    rho_t = torch.tensor(rho, device="cuda")
    T_t = torch.tensor(T, device="cuda")
    tgt = torch.tensor(target, device="cuda")

    def loss(d):
        with torch.no_grad():
            return float(temperature_loss(torch.tensor(d, device="cuda"), lat, rho_t, T_t, tgt, n, K))

    return [(loss(dT0 + eps * v) - loss(dT0 - eps * v)) / (2 * eps) for v in dirs]


def _directions(shape, k=16, seed=2024):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(shape) for _ in range(k)]


def test_rollout_gradient_matches_central_differences_16_directions():
    p, rho, T, target, dT0 = case(64, 96, seed=11)
    n, K = 200, 50
    _, g, _ = gpu_grad(p, rho, T, target, dT0, n, K)
    dirs = _directions(dT0.shape)
    fds = _fp64_central_differences(p, rho, T, target, dT0, n, K, dirs)
    worst = max(abs(fd - float((g * v).sum())) / abs(fd) for fd, v in zip(fds, dirs))
    assert worst <= 1e-6, worst


def test_fp32_store_rollout_gradient_matches_fp64_central_differences_16_directions():
    # The float32-store rollout's adjoint gradient against float64 central
    # differences of the float64 rollout: the bar of the adjoint (1e-6
    # relative) holds for the float32-store variant too.
    p, rho, T, target, dT0 = case(64, 96, seed=11)
    n, K = 200, 50
    _, g, _ = gpu_grad(p, rho, T, target, dT0, n, K, "fp32")
    dirs = _directions(dT0.shape)
    fds = _fp64_central_differences(p, rho, T, target, dT0, n, K, dirs)
    worst = max(abs(fd - float((g * v).sum())) / abs(fd) for fd, v in zip(fds, dirs))
    assert worst <= 1e-6, worst


def test_fp32_store_rollout_gradient_close_to_fp64():
    p, rho, T, target, dT0 = case(32, 48, seed=5)
    _, g64, _ = gpu_grad(p, rho, T, target, dT0, 40, 10, "fp64")
    _, g32, _ = gpu_grad(p, rho, T, target, dT0, 40, 10, "fp32")
    assert np.abs(g32 - g64).max() <= 1e-4 * np.abs(g64).max()


def test_fp64df_rollout_gradient_matches_oracle_adjoint():
    # double-float forward collide and cotangent sums (about 48 bits): the
    # float64 gradient bar of the oracle comparison still holds
    p, rho, T, target, dT0 = case(12, 16)
    n = 9
    J, g, _ = gpu_grad(p, rho, T, target, dT0, n, K=4, precision="fp64df")
    Jo = A.rollout_loss(dT0, rho, T, target, p, n)
    go = A.rollout_grad(dT0, rho, T, target, p, n)
    assert J == pytest.approx(Jo, rel=1e-12)
    assert np.abs(g - go).max() <= 1e-10 * np.abs(go).max()


def test_fp32_store_rollout_with_float32_cotangents():
    # Float32 cotangents round the cotangent field to float32 at every step;
    # over the 200 steps the rounding accumulates to about 1e-5 of the
    # gradient (measured 1.0e-5 against the float64 rollout's gradient, 3.8e-5
    # worst directional error against float64 central differences), against
    # 5e-8 and 2e-7 with float64 cotangents.  Bars: 1e-4 for both.
    p, rho, T, target, dT0 = case(64, 96, seed=11)
    n, K = 200, 50
    _, g64, _ = gpu_grad(p, rho, T, target, dT0, n, K)
    lat = Lattice(p.lx, p.ly, tau=p.tau, g=p.g, t_top=p.t_top, t_bottom=p.t_bottom, precision="fp32",
                  rho0=float(rho.mean()))
    d = torch.tensor(dT0, device="cuda", requires_grad=True)
    J = temperature_loss(d, lat, torch.tensor(rho, device="cuda"), torch.tensor(T, device="cuda"),
                         torch.tensor(target, device="cuda"), n, K, cotangent_dtype=torch.float32)
    J.backward()
    g = d.grad.cpu().numpy()
    assert np.abs(g - g64).max() <= 1e-4 * np.abs(g64).max()
    dirs = _directions(dT0.shape)
    fds = _fp64_central_differences(p, rho, T, target, dT0, n, K, dirs)
    worst = max(abs(fd - float((g * v).sum())) / abs(fd) for fd, v in zip(fds, dirs))
    assert worst <= 1e-4, worst
