"""Discrete adjoint of the D2Q37 step (oracle side; test infrastructure).

The paper has no adjoint; this is the exact transpose of the Jacobian of one
float64 time step of ``oracle.model``:  step = C o B o P  (collide after bc
after propagate, Sect. 2), so for a cotangent lam on the output

    lam_t = P^T B^T C^T lam_{t+1}.

* (B P)^T is written out by hand from the linear map B P: every slot that P
  fills by a pull is pushed back to its source; every slot that bc fills is
  M(x) q_l, so its cotangent reaches each lost population that makes up M(x).
* C^T is formed from the exact per-site Jacobian of collide, obtained by the
  complex-step derivative  dF/dx = Im F(x + i h) / h  (h = 1e-30; no
  subtractive cancellation, exact to rounding) in each of the 37 directions.

Readings for the adjoint study:
* loss J = mean over physical sites of (T_final - T_target)^2;
* the control is a per-site initial temperature perturbation dT0, with
  f_0 = f^eq(rho_0, 0, T_0 + dT0) and rho_0 held fixed.
"""
from __future__ import annotations

import numpy as np

from . import model as M

H_CS = 1e-30


def propagate_bc_transpose(mu, p: M.Params):
    """(B P)^T mu for mu of shape (37, ly+6, lx); halos of the result are NaN."""
    xi = M.K()["xi"]
    ly = p.ly
    H = M.HALO
    lam = np.full_like(mu, np.nan)
    for l in range(M.NPOP):
        ax, ay = int(xi[l, 0]), int(xi[l, 1])
        if p.periodic_y:
            src = mu[l, H:H + ly, :]
            lam[l, H:H + ly, :] = np.roll(np.roll(src, -ay, axis=0), -ax, axis=1)
            continue
        for y0 in range(ly):
            if 0 <= y0 + ay < ly:
                lam[l, H + y0, :] = np.roll(mu[l, H + y0 + ay, :], -ax)
    if p.periodic_y:
        return lam
    for wall, T_wall in (("bottom", p.t_bottom), ("top", p.t_top)):
        q = M.wall_q(T_wall, wall)
        Lam = 0.0
        for (d, l) in M.unknown_slots(wall):
            y = d if wall == "bottom" else ly - 1 - d
            Lam = Lam + q[l] * mu[l, H + y, :]
        for (l, y0) in M.lost_terms(wall, ly):
            lam[l, H + y0, :] = np.roll(Lam, -int(xi[l, 0]))
    return lam


def site_jacobian(fun, x):
    """Per-site Jacobian of a site-local map fun: (37, ...) -> (m, ...).

    Returns J of shape (m, 37, ...), J[k, l] = d fun_k / d x_l, by complex step.
    """
    cols = []
    for l in range(x.shape[0]):
        xc = x.astype(np.complex128)
        xc[l] += 1j * H_CS
        cols.append(np.imag(fun(xc)) / H_CS)
    return np.stack(cols, axis=1)


def collide_vjp(ft, lam, p: M.Params):
    """C^T lam at the post-bc state ft (both (37, ly+6, lx)); halos NaN."""
    fp = M.physical(ft)

    def coll(x):
        full = np.full((M.NPOP,) + ft.shape[1:], np.nan, dtype=x.dtype)
        full[:, M.HALO:-M.HALO] = x
        return M.physical(M.collide(full, p))

    J = site_jacobian(coll, fp)                       # (37 out, 37 in, ly, lx)
    out = np.full_like(ft, np.nan)
    out[:, M.HALO:-M.HALO] = np.einsum("kl...,k...->l...", J, M.physical(lam))
    return out


def adjoint_step(f_t, lam_next, p: M.Params):
    """lam_t = (B P)^T C^T lam_{t+1}, with C linearised at B P f_t."""
    return propagate_bc_transpose(collide_vjp(M.propagate_bc(f_t, p), lam_next, p), p)


def moments_vjp(f, g_rho, g_ux, g_uy, g_T):
    """sum over fields of (d field / d f)^T g_field, per site; f is (37, ly+6, lx)."""
    fp = M.physical(f)

    def mom(x):
        return np.stack(M.moments(x))

    J = site_jacobian(mom, fp)                         # (4, 37, ly, lx)
    g = np.stack([g_rho, g_ux, g_uy, g_T])
    out = np.full_like(f, np.nan)
    out[:, M.HALO:-M.HALO] = np.einsum("kl...,k...->l...", J, g)
    return out


def equilibrium_vjp(rho, ux, uy, T, lam):
    """Cotangents (g_rho, g_ux, g_uy, g_T) of sum_l lam_l f^eq_l(rho, u, T)."""
    lp = M.physical(lam)
    out = []
    base = [np.asarray(v, dtype=np.complex128) for v in (rho, ux, uy, T)]
    for i in range(4):
        args = [b.copy() for b in base]
        args[i] = args[i] + 1j * H_CS
        out.append((np.imag(M.equilibrium(*args)) / H_CS * lp).sum(axis=0))
    return tuple(out)


# --------------------------------------------------------------------------
# Rollout loss and its gradient with respect to the initial temperature
# --------------------------------------------------------------------------

def rollout_loss(dT0, rho0, T0, T_target, p: M.Params, n: int):
    """J(dT0) = mean (T_n - T_target)^2 with f_0 = f^eq(rho0, 0, T0 + dT0)."""
    z = np.zeros_like(rho0)
    f = M.init_state(rho0, z, z, T0 + dT0, dtype=np.result_type(dT0, np.float64))
    f = M.run(f, p, n)
    T = M.moments(M.physical(f))[3]
    d = T - T_target
    return (d * d).mean()


def rollout_grad(dT0, rho0, T0, T_target, p: M.Params, n: int):
    """dJ/d(dT0) by the discrete adjoint: store the trajectory, sweep back."""
    z = np.zeros_like(rho0)
    f = M.init_state(rho0, z, z, T0 + dT0)
    traj = [f]
    for _ in range(n):
        f = M.step(f, p)
        traj.append(f)
    T = M.moments(M.physical(f))[3]
    gT = 2.0 * (T - T_target) / T.size
    lam = moments_vjp(f, 0 * gT, 0 * gT, 0 * gT, gT)
    for t in range(n - 1, -1, -1):
        lam = adjoint_step(traj[t], lam, p)
    return equilibrium_vjp(rho0, z, z, T0 + dT0, lam)[3]
