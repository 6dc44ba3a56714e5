"""Checkpointed adjoint rollouts of the D2Q37 step as a torch.autograd.Function.

Forward: f_0 = f^eq(rho_0, 0, T_0 + dT0), n fused steps, output the final
temperature field T_n (eq. 2).  A copy of the state is kept every K steps.
Backward: the cotangent of T_n is mapped onto the populations
(lbm_moments_vjp); then, newest segment first, the segment's states are
recomputed from its checkpoint with lbm_step_from and the discrete adjoint
steps (lbm_adjoint_step) run back through them; finally the cotangent of f_0
is mapped to dT0 (lbm_init_vjp).  Memory: n / K checkpoints plus K states.

All arithmetic runs in liblbm.so; this module only orders the calls and owns
the buffers.
"""
from __future__ import annotations

import torch

from .lbm import Lattice


class TemperatureRollout(torch.autograd.Function):
    """T_n(dT0) for a fixed lattice (walls, tau, g) and fixed rho_0, T_0."""

    @staticmethod
    def forward(ctx, dT0: torch.Tensor, lattice: Lattice, rho0: torch.Tensor, T0: torch.Tensor,
                n: int, K: int, cotangent_dtype: torch.dtype = torch.float64):
        lat = lattice
        z = torch.zeros_like(rho0)
        Tin = (T0 + dT0.detach()).contiguous()
        lat.init(rho0, z, z, Tin)
        ckpts = []
        done = 0
        while done < n:
            ckpts.append(lat.state().clone())
            k = min(K, n - done)
            lat.step(k)
            done += k
        f_n = lat.state().clone()
        T_n = lat.moments(f_n)[3]
        ctx.lattice = lat
        ctx.n, ctx.K = n, K
        ctx.cot = cotangent_dtype
        ctx.ckpts = ckpts
        ctx.save_for_backward(rho0, Tin, f_n)
        return T_n

    @staticmethod
    def backward(ctx, gT: torch.Tensor):
        lat: Lattice = ctx.lattice
        rho0, Tin, f_n = ctx.saved_tensors
        n, K = ctx.n, ctx.K
        lam = lat.moments_vjp(f_n, None, None, None, gT.contiguous(), dtype=ctx.cot)
        lam_next = lat.new_cotangent(dtype=ctx.cot)
        seg_states = [lat.new_state() for _ in range(K)]
        nseg = len(ctx.ckpts)
        for s in range(nseg - 1, -1, -1):
            length = min(K, n - s * K)
            seg_states[0].copy_(ctx.ckpts[s])
            for t in range(1, length):
                lat.step_from(seg_states[t - 1], seg_states[t])
            for t in range(length - 1, -1, -1):
                lat.adjoint_step(seg_states[t], lam, lam_next)
                lam, lam_next = lam_next, lam
        z = torch.zeros_like(rho0)
        g = lat.init_vjp(rho0, z, z, Tin, lam)[3]
        ctx.ckpts = None
        return g, None, None, None, None, None, None


def temperature_loss(dT0, lattice: Lattice, rho0, T0, T_target, n: int, K: int = 50,
                     cotangent_dtype: torch.dtype = torch.float64):
    """J = mean over sites of (T_n - T_target)^2, differentiable in dT0.
    cotangent_dtype=torch.float32 runs the backward sweep with float32
    cotangents and the float32 adjoint (FP32-store lattices only)."""
    T_n = TemperatureRollout.apply(dT0, lattice, rho0, T0, n, K, cotangent_dtype)
    d = T_n - T_target
    return (d * d).mean()
