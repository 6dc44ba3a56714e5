"""Pins of the oracle's row-averaged observables (CPU only)."""
import numpy as np
import pytest

import synth
from oracle import model as M, observables as O


def test_uniform_state_gives_its_own_values():
    lx, ly = 6, 9
    rho, ux, uy, T = 1.3, 0.04, -0.02, 0.9
    f = M.init_state(np.full((ly, lx), rho), np.full((ly, lx), ux), np.full((ly, lx), uy), np.full((ly, lx), T))
    prof = O.profiles(f, M.Params(lx, ly, tau=0.8, g=0.0))
    want = [rho, ux, uy, T, T * T, uy * T, 0.5 * rho * (ux * ux + uy * uy), rho * uy]
    for i, w in enumerate(want):
        np.testing.assert_allclose(prof[i], w, rtol=1e-13, atol=1e-16)


def test_free_fall_midpoint_velocity():
    # a uniform periodic fluid at rest falls freely: after n steps the
    # hydrodynamic velocity is the mid-step velocity -(n - 1/2) g.
    lx, ly, g = 5, 6, 1e-3
    z = np.zeros((ly, lx))
    f = M.init_state(z + 1.1, z, z, z + 1.0)
    p = M.Params(lx, ly, tau=0.7, g=g, periodic_y=True)
    for n in range(1, 4):
        f = M.step(f, p)
        prof = O.profiles(f, p)
        np.testing.assert_allclose(prof[2], -(n - 0.5) * g, rtol=1e-12)
        np.testing.assert_allclose(prof[7], -1.1 * (n - 0.5) * g, rtol=1e-12)


def test_heat_flux_and_kinetic_energy_vanish_at_rest():
    rho, ux, uy, T, tt, tb = synth.rt_fields(16, 12, 3, 1)
    f = M.init_state(rho, ux, uy, T)
    prof = O.profiles(f, M.Params(16, 12, tau=0.8, g=0.0, t_top=tt, t_bottom=tb))
    np.testing.assert_allclose(prof[5], 0.0, atol=1e-15)
    np.testing.assert_allclose(prof[6], 0.0, atol=1e-15)
    # the temperature profile is the x-average of the initial field
    np.testing.assert_allclose(prof[3], T.mean(axis=1), rtol=1e-13)
