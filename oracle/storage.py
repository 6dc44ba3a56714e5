"""Float32 shifted storage of the populations (oracle side; test infrastructure).

Not in the paper, whose populations are float64 throughout (Sect. 4 counts
8-byte populations).  It is a storage format of this library that halves the
bytes a time step moves: population l is held as the float32 deviation

    d_l = fl32(f_l - w_l rho0)          (round to nearest even)

from a fixed density rho0, and read back as f_l = w_l rho0 + d_l (the float64
sum, one rounding).  w_l rho0 is the float64 product of the weight and rho0.

``step_fp32_storage`` is the float64 oracle step of ``oracle.model`` between a
decode and an encode: its distance from the float64 oracle is the error of the
storage alone, the floor that no float32-storage arithmetic can go below.
"""
from __future__ import annotations

import numpy as np

from . import lattice, model

HALO = model.HALO


def _w_rho0(rho0):
    return (lattice.constants()["w"] * float(rho0))[:, None, None]


def encode(f, rho0):
    """float32 deviations of a float64 state (37, ly + 6, lx); halos stay NaN."""
    d = np.full(f.shape, np.nan, dtype=np.float32)
    d[:, HALO:-HALO] = (f[:, HALO:-HALO] - _w_rho0(rho0)).astype(np.float32)
    return d


def decode(d, rho0):
    """float64 populations w_l rho0 + d_l of a float32 deviation state."""
    return d.astype(np.float64) + _w_rho0(rho0)


def step_fp32_storage(d, p: model.Params, rho0):
    """One oracle time step (propagate, bc, collide; Sect. 2, eq. (1)) on the
    decoded populations, stored back as float32 deviations."""
    return encode(model.step(decode(d, rho0), p), rho0)


def run_fp32_storage(d, p: model.Params, rho0, n: int):
    for _ in range(n):
        d = step_fp32_storage(d, p, rho0)
    return d
