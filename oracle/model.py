"""D2Q37 thermal BGK time step: plain float64 oracle (test infrastructure).

Follows the paper's statement of the model and its three kernels:

* eq. (1), the BGK evolution  f_l(x, t+1) = f_l(x - c_l, t)
  - (1/tau) (f_l(x - c_l, t) - f_l^eq), with Delta t = 1 (Sect. 2);
* eq. (2), the macroscopic fields  rho = sum f,  rho u = sum c f,
  D rho T = sum |c - u|^2 f  (Sect. 2);
* the time step as propagate, then bc, then collide (Sect. 2, bullet list),
  with periodic left/right edges (Sect. 2, "For the left and right edges");
* the SoA layout: each population's plane is contiguous (Fig. "streamscheme",
  Sect. 4).

State layout (shared interface with the library, documented in its header):
``f[l, y + 3, x]`` for l in 0..36, y in -3..ly+2 (three halo rows below and
above the ly physical rows), x in 0..lx-1 periodic.  Halo rows are never read
as data; the oracle fills them with NaN so that any leak shows.

Readings where the paper is silent:

1. Equilibrium: the 4th-order Hermite expansion of the Maxwellian about the
   lattice reference temperature 1 (theta = T - 1):
   f^eq_l = w_l rho sum_{n<=4} a^(n)(u, theta) : H^(n)(c_l) / n!.
   The paper only says the equilibria are known functions of rho, u, T and
   mentions a Hermite projection (Sect. 2).  Two forms are given below: the
   explicit tensor sum and its expansion in c.u, |u|^2, |c|^2, theta.
2. Collide is plain BGK, eq. (1), Delta t = 1, omega = 1/tau.
3. Gravity g along -y enters as an equilibrium shift: the equilibrium is taken
   at u' = u + tau g and T' = T + tau (1 - tau) |g|^2 / D.  Per collide this
   adds rho g to the momentum and leaves rho and T unchanged.
4. bc at the top and bottom walls (fixed temperature, zero velocity; Sect. 2,
   bc bullet): a diffuse thermal wall with per-column mass balance.  After
   propagate, each slot (x, y, l) whose pull source lies in a halo row is
   "unknown" (26 per column per wall).  It is set to M(x) q_l, where M(x) is
   the mass that left the lattice through that wall during propagate and
   would have landed in column x, and q_l = phi_l / sum_slots phi with
   phi_l = f^eq_l(1, 0, T_wall).  M(x) is summed in a fixed order: l
   ascending, then source row ascending.  q_l is the float64 nearest to the
   exact value (computed in 60-digit decimal arithmetic).
5. Periodic left/right edges by modular indexing on one lattice (the halo
   columns and their copy are an MPI-era device of Sect. 4).
"""
from __future__ import annotations

import dataclasses
from decimal import Decimal, getcontext

import numpy as np

from . import lattice

D = lattice.D
NPOP = lattice.NPOP
HALO = 3


@dataclasses.dataclass
class Params:
    lx: int
    ly: int
    tau: float
    g: float = 0.0          # gravity magnitude, acting along -y
    t_top: float = 1.0
    t_bottom: float = 1.0
    periodic_y: bool = False  # test mode: no walls, y periodic


def K():
    return lattice.constants()


# --------------------------------------------------------------------------
# Equilibrium
# --------------------------------------------------------------------------

def equilibrium(rho, ux, uy, T):
    """Closed form of the 4th-order Hermite equilibrium; returns (37, *shape).

    With cu = c_l.u, u2 = |u|^2, c2 = |c_l|^2, theta = T - 1:
      P = 1 + cu + 1/2 [cu^2 - u2 + theta (c2 - D)]
            + cu/6 [cu^2 - 3 u2 + 3 theta (c2 - D - 2)]
            + 1/24 [cu^4 - 6 cu^2 u2 + 3 u2^2
                    + 6 theta (cu^2 (c2 - D - 4) + u2 (D + 2 - c2))
                    + 3 theta^2 (c2^2 - 2 (D + 2) c2 + D (D + 2))]
      f^eq_l = w_l rho P.
    """
    k = K()
    rho, ux, uy, T = np.broadcast_arrays(rho, ux, uy, T)
    theta = T - 1.0
    u2 = ux * ux + uy * uy
    out = []
    for l in range(NPOP):
        cx, cy = k["c"][l]
        c2 = k["c2"][l]
        cu = cx * ux + cy * uy
        p = (1.0 + cu
             + 0.5 * (cu * cu - u2 + theta * (c2 - D))
             + cu / 6.0 * (cu * cu - 3.0 * u2 + 3.0 * theta * (c2 - D - 2))
             + (cu ** 4 - 6.0 * cu * cu * u2 + 3.0 * u2 * u2
                + 6.0 * theta * (cu * cu * (c2 - D - 4) + u2 * (D + 2 - c2))
                + 3.0 * theta * theta * (c2 * c2 - 2 * (D + 2) * c2 + D * (D + 2))) / 24.0)
        out.append(k["w"][l] * rho * p)
    return np.stack(out)


def _hermite_tensors(c):
    """H^(0..4)(c) for one 2-vector c (tensor Hermite polynomials, unit variance)."""
    I = np.eye(D)
    H1 = np.array(c, dtype=np.float64)
    H2 = np.einsum("i,j->ij", H1, H1) - I
    H3 = (np.einsum("i,j,k->ijk", H1, H1, H1)
          - np.einsum("i,jk->ijk", H1, I) - np.einsum("j,ik->ijk", H1, I)
          - np.einsum("k,ij->ijk", H1, I))
    cc = np.einsum("i,j->ij", H1, H1)
    H4 = (np.einsum("i,j,k,l->ijkl", H1, H1, H1, H1)
          - np.einsum("ij,kl->ijkl", cc, I) - np.einsum("ik,jl->ijkl", cc, I)
          - np.einsum("il,jk->ijkl", cc, I) - np.einsum("jk,il->ijkl", cc, I)
          - np.einsum("jl,ik->ijkl", cc, I) - np.einsum("kl,ij->ijkl", cc, I)
          + np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I)
          + np.einsum("il,jk->ijkl", I, I))
    return H1, H2, H3, H4


def equilibrium_hermite(rho, ux, uy, T):
    """Explicit tensor form f^eq_l = w_l rho sum_n a^(n) : H^(n)(c_l) / n!.

    Maxwellian Hermite coefficients per unit density (theta = T - 1):
      a1 = u, a2 = uu + theta I, a3 = uuu + theta sym3(u I),
      a4 = uuuu + theta sym6(uu I) + theta^2 sym3(I I).
    """
    k = K()
    rho, ux, uy, T = np.broadcast_arrays(rho, ux, uy, T)
    theta = T - 1.0
    u = np.stack([ux, uy], axis=-1)                       # (..., 2)
    I = np.eye(D)
    uu = np.einsum("...i,...j->...ij", u, u)
    a2 = uu + theta[..., None, None] * I
    sym3_uI = (np.einsum("...i,jk->...ijk", u, I) + np.einsum("...j,ik->...ijk", u, I)
               + np.einsum("...k,ij->...ijk", u, I))
    a3 = np.einsum("...i,...j,...k->...ijk", u, u, u) + theta[..., None, None, None] * sym3_uI
    sym6_uuI = (np.einsum("...ij,kl->...ijkl", uu, I) + np.einsum("...ik,jl->...ijkl", uu, I)
                + np.einsum("...il,jk->...ijkl", uu, I) + np.einsum("...jk,il->...ijkl", uu, I)
                + np.einsum("...jl,ik->...ijkl", uu, I) + np.einsum("...kl,ij->...ijkl", uu, I))
    sym3_II = (np.einsum("ij,kl->ijkl", I, I) + np.einsum("ik,jl->ijkl", I, I)
               + np.einsum("il,jk->ijkl", I, I))
    t4 = theta[..., None, None, None, None]
    a4 = (np.einsum("...i,...j,...k,...l->...ijkl", u, u, u, u) + t4 * sym6_uuI
          + t4 * t4 * sym3_II)
    out = []
    for l in range(NPOP):
        H1, H2, H3, H4 = _hermite_tensors(k["c"][l])
        p = (1.0 + np.einsum("...i,i->...", u, H1)
             + np.einsum("...ij,ij->...", a2, H2) / 2.0
             + np.einsum("...ijk,ijk->...", a3, H3) / 6.0
             + np.einsum("...ijkl,ijkl->...", a4, H4) / 24.0)
        out.append(k["w"][l] * rho * p)
    return np.stack(out)


# --------------------------------------------------------------------------
# Macroscopic fields, eq. (2)
# --------------------------------------------------------------------------

def moments(fp):
    """eq. (2) on populations fp of shape (37, ...): returns rho, ux, uy, T."""
    k = K()
    rho = fp.sum(axis=0)
    jx = np.tensordot(k["c"][:, 0], fp, axes=(0, 0))
    jy = np.tensordot(k["c"][:, 1], fp, axes=(0, 0))
    ux = jx / rho
    uy = jy / rho
    e = 0.0
    for l in range(NPOP):
        dx = k["c"][l, 0] - ux
        dy = k["c"][l, 1] - uy
        e = e + (dx * dx + dy * dy) * fp[l]
    T = e / (D * rho)
    return rho, ux, uy, T


def physical(f):
    """View of the physical rows of a (37, ly+6, lx) state."""
    return f[:, HALO:-HALO, :]


def init_state(rho, ux, uy, T, dtype=np.float64):
    """Populations at equilibrium f^eq(rho, u, T), halos NaN; fields are (ly, lx)."""
    ly, lx = np.shape(rho)
    f = np.full((NPOP, ly + 2 * HALO, lx), np.nan, dtype=dtype)
    f[:, HALO:-HALO, :] = equilibrium(rho, ux, uy, T)
    return f


# --------------------------------------------------------------------------
# propagate, bc, collide (Sect. 2 bullet list)
# --------------------------------------------------------------------------

def propagate(f, p: Params):
    """Pull every population from x - c_l (eq. (1) first term; Fig. "propagate").

    out[l, y, x] = f[l, y - xi_ly, (x - xi_lx) mod lx] for physical y.  With
    walls the source row may be a halo row (those slots are replaced by bc);
    in periodic_y mode the source row wraps modulo ly.  Output halos are NaN.
    """
    xi = K()["xi"]
    ly = p.ly
    out = np.full_like(f, np.nan)
    for l in range(NPOP):
        ax, ay = int(xi[l, 0]), int(xi[l, 1])
        if p.periodic_y:
            src = np.roll(f[l, HALO:HALO + ly, :], ay, axis=0)
        else:
            src = f[l, HALO - ay:HALO + ly - ay, :]
        out[l, HALO:HALO + ly, :] = np.roll(src, ax, axis=1)
    return out


def _phi(T_wall):
    """phi_l = f^eq_l(1, 0, T_wall) in 60-digit decimals, for all l."""
    k = K()
    getcontext().prec = 60
    y = k["y_dec"]
    th = Decimal(float(T_wall)) - 1
    out = []
    for l in range(NPOP):
        s = int(k["shell"][l])
        c2 = Decimal(s) / y
        w = k["w_dec"][s]
        out.append(w * (1 + th * (c2 - D) / 2 + th * th * (c2 * c2 - 2 * (D + 2) * c2 + D * (D + 2)) / 8))
    return out


def unknown_slots(wall: str):
    """Unknown (row offset from the wall, l) pairs: rows 0..2 from the wall whose
    pull source lies beyond it.  'bottom' rows are y = 0, 1, 2; 'top' rows are
    y = ly-1, ly-2, ly-3 (offset d means y = ly-1-d)."""
    xi = K()["xi"]
    out = []
    for d in range(3):
        for l in range(NPOP):
            vy = int(xi[l, 1]) if wall == "bottom" else -int(xi[l, 1])
            if vy > d:
                out.append((d, l))
    return out


def wall_q(T_wall, wall: str):
    """q_l = phi_l / sum over the wall's 26 unknown slots of phi (float64 nearest)."""
    phi = _phi(T_wall)
    slots = unknown_slots(wall)
    tot = sum(phi[l] for (_, l) in slots)
    q = np.zeros(NPOP)
    for (_, l) in slots:
        q[l] = float(phi[l] / tot)
    return q


def lost_terms(wall: str, ly: int):
    """(l, source row y0) pairs whose propagate target lies beyond the wall, in
    the canonical summation order: l ascending, then y0 ascending."""
    xi = K()["xi"]
    out = []
    for l in range(NPOP):
        vy = int(xi[l, 1])
        rows = range(0, 3) if wall == "bottom" else range(ly - 3, ly)
        for y0 in rows:
            if (wall == "bottom" and y0 + vy < 0) or (wall == "top" and y0 + vy >= ly):
                out.append((l, y0))
    return out


def bc(fprop, fpre, p: Params):
    """Thermal-wall bc after propagate (reading 4 above); returns a new array."""
    if p.periodic_y:
        return fprop.copy()
    xi = K()["xi"]
    out = fprop.copy()
    ly = p.ly
    for wall, T_wall in (("bottom", p.t_bottom), ("top", p.t_top)):
        q = wall_q(T_wall, wall)
        M = None
        for (l, y0) in lost_terms(wall, ly):
            # source column x - xi_lx lands in column x
            term = np.roll(fpre[l, HALO + y0, :], int(xi[l, 0]))
            M = term.copy() if M is None else M + term
        for (d, l) in unknown_slots(wall):
            y = d if wall == "bottom" else ly - 1 - d
            out[l, HALO + y, :] = M * q[l]
    return out


def collide(ft, p: Params):
    """BGK collide of eq. (1) on the physical rows of ft (reading 3 for gravity)."""
    out = np.full_like(ft, np.nan)
    fp = physical(ft)
    rho, ux, uy, T = moments(fp)
    uys = uy - p.tau * p.g
    Ts = T + p.tau * (1.0 - p.tau) * p.g * p.g / D
    feq = equilibrium(rho, ux, uys, Ts)
    out[:, HALO:-HALO, :] = fp - (fp - feq) / p.tau
    return out


# --------------------------------------------------------------------------
# Regularised collide (the Hermite projection the paper mentions, Sect. 2)
# --------------------------------------------------------------------------

def _hermite_stack():
    """H^(1..4)(c_l) for all l, as arrays (37, 2), (37, 2, 2), (37, 2, 2, 2), (37, 2, 2, 2, 2)."""
    k = K()
    hs = [_hermite_tensors(k["c"][l]) for l in range(NPOP)]
    return [np.stack([h[i] for h in hs]) for i in range(4)]


def hermite_project(fp):
    """Projection onto the Hermite polynomials of order <= 4 (weight w):
    (Pi f)_l = w_l sum_{n<=4} a^(n) : H^(n)(c_l) / n!,  a^(n) = sum_m f_m H^(n)(c_m).
    fp has shape (37, ...)."""
    H1, H2, H3, H4 = _hermite_stack()
    a0 = fp.sum(axis=0)
    a1 = np.einsum("p...,pi->...i", fp, H1)
    a2 = np.einsum("p...,pij->...ij", fp, H2)
    a3 = np.einsum("p...,pijk->...ijk", fp, H3)
    a4 = np.einsum("p...,pijkm->...ijkm", fp, H4)
    out = (a0[None]
           + np.einsum("...i,pi->p...", a1, H1)
           + np.einsum("...ij,pij->p...", a2, H2) / 2.0
           + np.einsum("...ijk,pijk->p...", a3, H3) / 6.0
           + np.einsum("...ijkm,pijkm->p...", a4, H4) / 24.0)
    w = K()["w"].reshape((NPOP,) + (1,) * (fp.ndim - 1))
    return w * out


def collide_regularized(ft, p: Params):
    """Regularised BGK: the non-equilibrium part is projected onto the order-<=4
    Hermite space before relaxing,
      f <- f^eq + (1 - 1/tau) Pi(f - f^eq),
    with the same moments, gravity shift and equilibrium as collide().  Pi keeps
    every moment of order <= 4, so mass, momentum (+ rho g) and energy change
    exactly as in plain BGK; the components outside the Hermite space are
    removed instead of relaxed."""
    out = np.full_like(ft, np.nan)
    fp = physical(ft)
    rho, ux, uy, T = moments(fp)
    uys = uy - p.tau * p.g
    Ts = T + p.tau * (1.0 - p.tau) * p.g * p.g / D
    feq = equilibrium(rho, ux, uys, Ts)
    out[:, HALO:-HALO, :] = feq + (1.0 - 1.0 / p.tau) * hermite_project(fp - feq)
    return out


def step_regularized(f, p: Params):
    return collide_regularized(propagate_bc(f, p), p)


def propagate_bc(f, p: Params):
    return bc(propagate(f, p), f, p)


def step(f, p: Params):
    """One time step: propagate, then bc, then collide (Sect. 2)."""
    return collide(propagate_bc(f, p), p)


def run(f, p: Params, n: int):
    for _ in range(n):
        f = step(f, p)
    return f
