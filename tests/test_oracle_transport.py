"""Transport pins of the oracle's step: decay rates from kinetic theory (CPU only).

The paper's model is a thermal LB scheme for the hydrodynamic equations with
heat transport (Sect. 2).  For the BGK collision of eq. (1) with Delta t = 1,
the Chapman-Enskog expansion gives the kinematic viscosity nu = T (tau - 1/2)
and the thermal diffusivity chi = nu (the BGK Prandtl number is 1), in the
units where the discrete velocities are c = r xi; one lattice site is r of
those length units, so in site units both are divided by r^2.  On a fully
periodic lattice a small sinusoidal mode of wavenumber k = 2 pi / Ly then
decays as exp(-nu k^2 t):

* a shear wave u_x = U sin(k y) at uniform rho and T, at rate nu k^2;
* an isobaric temperature wave (rho T = const, u = 0), measured through the
  entropy fluctuation ds = (D/2) dT/T - drho/rho, at rate chi k^2 (the
  acoustic modes it also excites carry no entropy to linear order, so they
  drop out of ds).

* a density wave at uniform T, whose velocity mode oscillates at the
  adiabatic sound speed c_s = sqrt(gamma T) with gamma = (D + 2) / D = 2 (an
  isothermal scheme would give sqrt(T), 29 % lower).

The rates are measured between steps 50 and 250 on a 4 x 64 lattice and
agree with theory to about 0.3 % (the residual falls as k^2 with finer
waves); the tolerance is 0.5 %.  The sound frequency, from the zero
crossings of the velocity mode over 400 steps, agrees to 0.2 %.  The temperatures away from the reference
T = 1 make the theta-dependent terms of the equilibrium take part.
"""
import numpy as np
import pytest

from oracle import lattice, model as M, observables as O

R = lattice.constants()["r"]
LX, LY, T1, T2 = 4, 64, 50, 250
TOL = 5e-3


def _decay_rate(f, p, observe):
    """Decay rate per step of the sin(k y) component of observe(fields)."""
    s = np.sin(2 * np.pi * np.arange(LY) / LY)[:, None]
    amp = {}
    for t in range(1, T2 + 1):
        f = M.step(f, p)
        if t in (T1, T2):
            q = observe(M.moments(M.physical(f)))
            amp[t] = float((q * s).sum() / (s * s).sum())
    return np.log(amp[T1] / amp[T2]) / (T2 - T1)


def _theory(tau, T0):
    return T0 * (tau - 0.5) / R ** 2 * (2 * np.pi / LY) ** 2


@pytest.mark.parametrize("tau,T0", [(0.6, 1.0), (0.8, 0.7), (1.0, 1.25)])
def test_shear_wave_decays_at_the_bgk_viscosity(tau, T0):
    z = np.zeros((LY, LX))
    s = np.sin(2 * np.pi * np.arange(LY) / LY)[:, None] + z
    f = M.init_state(z + 1.0, 1e-4 * s, z, z + T0)
    p = M.Params(LX, LY, tau=tau, g=0.0, periodic_y=True)
    rate = _decay_rate(f, p, lambda m: m[1])
    assert abs(rate / _theory(tau, T0) - 1) < TOL, rate / _theory(tau, T0) - 1


@pytest.mark.parametrize("tau,T0", [(0.6, 1.0), (0.8, 0.7), (1.0, 1.25)])
def test_entropy_wave_decays_at_the_bgk_thermal_diffusivity(tau, T0):
    z = np.zeros((LY, LX))
    s = np.sin(2 * np.pi * np.arange(LY) / LY)[:, None] + z
    T = T0 * (1.0 + 1e-4 * s)
    f = M.init_state(1.0 / T, z, z, T)
    p = M.Params(LX, LY, tau=tau, g=0.0, periodic_y=True)

    def entropy(m):
        rho, _, _, temp = m
        return (M.D / 2) * (temp - temp.mean()) / temp.mean() - (rho - rho.mean()) / rho.mean()

    rate = _decay_rate(f, p, entropy)
    assert abs(rate / _theory(tau, T0) - 1) < TOL, rate / _theory(tau, T0) - 1


@pytest.mark.parametrize("tau,T0", [(0.6, 1.0), (1.0, 0.7)])
def test_density_wave_oscillates_at_the_adiabatic_sound_speed(tau, T0):
    z = np.zeros((LY, LX))
    y = np.arange(LY)[:, None] + z
    c, s = np.cos(2 * np.pi * y / LY), np.sin(2 * np.pi * y / LY)
    f = M.init_state(1.0 + 1e-4 * s, z, z, z + T0)
    p = M.Params(LX, LY, tau=tau, g=0.0, periodic_y=True)
    a = []
    for _ in range(400):
        f = M.step(f, p)
        a.append(float((M.moments(M.physical(f))[2] * c).sum() / (c * c).sum()))
    zero = [i + a[i] / (a[i] - a[i + 1]) for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    assert len(zero) >= 10
    omega = np.pi / np.diff(zero).mean()
    cs = np.sqrt((M.D + 2) / M.D * T0) / R
    assert abs(omega / (cs * 2 * np.pi / LY) - 1) < TOL, omega / (cs * 2 * np.pi / LY) - 1


@pytest.mark.parametrize("tau,g,T0", [(0.8, 1e-3, 1.0), (1.0, 1e-3, 1.2)])
def test_gravity_between_isothermal_walls_settles_into_the_isothermal_atmosphere(tau, g, T0):
    # Walls at one temperature T0 and gravity g along -y: the steady state is
    # hydrostatic, dp/dy = -rho g with p = rho T0, so rho ~ exp(-g y / T0)
    # (y in the length units of c = r xi: a slope of -g r / T0 per site), at
    # rest (mid-step velocity zero) and at the walls' temperature.  Checked in
    # the bulk rows after 1500 steps (settled to about 0.3 %).
    ly, lx = 32, 4
    z = np.zeros((ly, lx))
    f = M.init_state(z + 1.0, z, z, z + T0)
    p = M.Params(lx, ly, tau=tau, g=g, t_top=T0, t_bottom=T0)
    for _ in range(1500):
        f = M.step(f, p)
    rho, ux, uy_mid, T = O.fields(f, p)
    bulk = slice(8, ly - 8)
    slope = np.polyfit(np.arange(ly)[bulk], np.log(rho.mean(axis=1))[bulk], 1)[0]
    assert abs(slope / (-g * R / T0) - 1) < 1e-2, slope / (-g * R / T0) - 1
    assert np.abs(uy_mid[bulk]).max() < 1e-2 * g / 2
    assert np.abs(ux).max() < 1e-12
    assert np.abs(T[bulk] / T0 - 1).max() < 1e-3
