"""Row-averaged observables of a D2Q37 state (oracle side; test infrastructure).

The paper's codes run measurement routines that compute averages or
correlations of physical observables every few hundred or thousand steps
(Sect. 2).  The set used here, per physical row y, averaged over x:

  0 rho,  1 u_x,  2 u_y,  3 T,  4 T^2,  5 u_y T,  6 rho |u|^2 / 2,  7 rho u_y

with the macroscopic fields of eq. (2) and the hydrodynamic velocity
u = (sum c f - rho g_vec / 2) / rho, g_vec = (0, -g), of the stored
(post-collide) populations: with the equilibrium-shift force their first
moment already contains the whole impulse rho g_vec of the step, and removing
half of it gives the velocity at the midpoint of the step.
"""
from __future__ import annotations

import numpy as np

from . import model as M

NOBS = 8
NAMES = ("rho", "ux", "uy", "T", "T2", "uyT", "ekin", "rho_uy")


def fields(f, p: M.Params):
    """rho, hydrodynamic u_x, u_y, T on the physical rows (ly, lx)."""
    rho, ux, uy, T = M.moments(M.physical(f))
    return rho, ux, uy + 0.5 * p.g, T


def profiles(f, p: M.Params):
    """(8, ly) array of row averages of the observables listed above."""
    rho, ux, uy, T = fields(f, p)
    obs = [rho, ux, uy, T, T * T, uy * T, 0.5 * rho * (ux * ux + uy * uy), rho * uy]
    return np.stack([o.mean(axis=1) for o in obs])
