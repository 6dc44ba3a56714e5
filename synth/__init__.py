"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark.

This module holds no arithmetic of the lattice Boltzmann method itself: it only
draws macroscopic fields (density, velocity, temperature) and noise arrays from
``numpy.random.default_rng(seed)``.  Populations are built from these fields by
each side on its own (the oracle in ``oracle/``, the CUDA path in its kernels).

Workloads
---------
* ``rt_fields``: a Rayleigh-Taylor-like initial condition.  The paper runs its
  D2Q37 code on synthetic lattices for convective-turbulence studies (Sect. 2
  and Sect. 4, lattices such as 1920x2048); it gives no initial condition, so
  this one is stated here: a cold dense layer above a hot light layer,
  separated by a thin interface whose height is a sum of seeded cosines, in
  pressure balance (rho * T = p0) and at rest.
* ``random_fields`` / ``noise``: smooth-free random fields for one-step parity
  tests, exercising every velocity- and temperature-dependent term.
* ``batch_lattices``: a seeded list of independent lattices of uneven sizes
  and parameters.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

NPOP = 37
HALO = 3


def rt_fields(lx: int, ly: int, modes: int, seed: int, delta: float = 1.0,
              width: float = 1.0, p0: float = 1.0, amp_max: float = 2.0):
    """Rayleigh-Taylor-like fields on the physical lattice, shape (ly, lx).

    T(x, y) = 1 - (delta/2) * tanh((y - y_i(x)) / width), so the upper layer is
    cold (T = 1 - delta/2) and the lower one hot (T = 1 + delta/2);
    y_i(x) = ly/2 + sum_m A_m cos(2 pi k_m x / lx + phi_m) with A_m ~ U(0, amp_max),
    k_m distinct integers in [1, max(1, lx // 4)], phi_m ~ U(0, 2 pi);
    rho = p0 / T (isobaric, so the cold layer is the dense one); u = 0.

    Returns (rho, ux, uy, T, t_top, t_bottom) with the wall temperatures equal
    to the far-field temperatures of the adjacent layers.
    """
    rng = np.random.default_rng(seed)
    kmax = max(1, lx // 4)
    m = min(modes, kmax)
    ks = rng.choice(np.arange(1, kmax + 1), size=m, replace=False)
    amps = rng.uniform(0.0, amp_max, size=m)
    phis = rng.uniform(0.0, 2.0 * math.pi, size=m)
    x = np.arange(lx, dtype=np.float64)
    yi = np.full(lx, ly / 2.0)
    for k, a, ph in zip(ks, amps, phis):
        yi += a * np.cos(2.0 * math.pi * k * x / lx + ph)
    y = np.arange(ly, dtype=np.float64)[:, None]
    T = 1.0 - 0.5 * delta * np.tanh((y - yi[None, :]) / width)
    rho = p0 / T
    ux = np.zeros((ly, lx))
    uy = np.zeros((ly, lx))
    return (np.ascontiguousarray(rho), ux, uy, np.ascontiguousarray(T),
            1.0 - 0.5 * delta, 1.0 + 0.5 * delta)


def random_fields(lx: int, ly: int, seed: int, umax: float = 0.1,
                  rho_range=(0.7, 1.5), t_range=(0.7, 1.3)):
    """Independent uniform random (rho, ux, uy, T) per site, shape (ly, lx)."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(*rho_range, size=(ly, lx))
    ux = rng.uniform(-umax, umax, size=(ly, lx))
    uy = rng.uniform(-umax, umax, size=(ly, lx))
    T = rng.uniform(*t_range, size=(ly, lx))
    return rho, ux, uy, T


def noise(lx: int, ly: int, seed: int, shape_prefix=(NPOP,)):
    """Uniform(-1, 1) noise of shape (*shape_prefix, ly, lx)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=tuple(shape_prefix) + (ly, lx))


def smooth_field(lx: int, ly: int, seed: int, modes: int = 6, amp: float = 0.1):
    """A smooth periodic-in-x random field (sum of seeded 2-D cosines), (ly, lx)."""
    rng = np.random.default_rng(seed)
    x = np.arange(lx)[None, :] / lx
    y = np.arange(ly)[:, None] / ly
    out = np.zeros((ly, lx))
    for _ in range(modes):
        kx = rng.integers(1, 4)
        ky = rng.integers(1, 4)
        a = rng.uniform(-amp, amp)
        ph = rng.uniform(0, 2 * math.pi, size=2)
        out += a * np.cos(2 * math.pi * kx * x + ph[0]) * np.cos(math.pi * ky * y + ph[1])
    return out


@dataclasses.dataclass
class LatticeSpec:
    lx: int
    ly: int
    tau: float
    g: float
    delta: float
    seed: int


def batch_lattices(n: int, seed: int,
                   lx_choices=(128, 256, 512, 1024),
                   ly_choices=(256, 512, 1024, 2048),
                   tau_range=(0.55, 1.0), g_range=(1e-5, 1e-4),
                   delta_range=(0.2, 1.0)):
    """n independent lattices with seeded uneven sizes and parameters."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(LatticeSpec(
            lx=int(rng.choice(lx_choices)), ly=int(rng.choice(ly_choices)),
            tau=float(rng.uniform(*tau_range)), g=float(rng.uniform(*g_range)),
            delta=float(rng.uniform(*delta_range)),
            seed=int(rng.integers(0, 2**31 - 1))))
    return out
