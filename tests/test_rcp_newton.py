"""The float64 step's 1/rho (rcp_nr in lbm_device.cuh), emulated word by word
with Python integers and exact rationals (CPU only).

The method is the Newton-Raphson iteration for the reciprocal taken to third
order in one step: from a seed y0 with e = 1 - x y0, y0 (1 + e + e^2) equals
(1 - e^3) / x.  The seed is x's top 23 significand bits as a float32
(integer operations), a float32 reciprocal approximation of that (modelled
here by every float32 within 4 units of the correctly rounded reciprocal,
more than the approximation's documented error), and its exact widening to
float64 (integer operations).  Claims checked:
  * the float32 built from x's bits is x truncated to 24 significant bits,
    and the widening reproduces the float32 exactly;
  * the result is within one unit in the last place of 1/x for x in
    [2^-125, 2^126), whatever seed of that quality the approximation gives;
  * x outside that range (zero, subnormals, infinities, NaN) gives NaN.
"""
import math
import struct
from fractions import Fraction

import numpy as np

M32 = 0xFFFFFFFF


def words(v):
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    return b >> 32, b & M32


def from_words(hi, lo):
    return struct.unpack("<d", struct.pack("<Q", ((hi & M32) << 32) | (lo & M32)))[0]


def f32_bits(v):
    return struct.unpack("<I", struct.pack("<f", v))[0]


def f32_from_bits(b):
    return struct.unpack("<f", struct.pack("<I", b & M32))[0]


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def seed_float(x):
    """The float32 operand of the reciprocal approximation, from x's words."""
    hi, lo = words(x)
    ex = ((hi >> 20) & 0x7FF) - 1023
    xf = (hi & 0x80000000) | (((ex + 127) << 23) & M32) | ((hi & 0xFFFFF) << 3) | (lo >> 29)
    return ex, f32_from_bits(xf & M32)


def widen(rf):
    rb = f32_bits(rf)
    yhi = (rb & 0x80000000) | ((((rb >> 23) & 0xFF) + (1023 - 127)) << 20) | ((rb & 0x7FFFFF) >> 3)
    return from_words(yhi, (rb << 29) & M32)


def rcp_nr(x, seed_ulps):
    """The device steps, with the approximation returning the float32 that
    lies seed_ulps units from the correctly rounded reciprocal."""
    ex, xf = seed_float(x)
    r = np.float32(1.0) / np.float32(xf) if xf != 0 else np.float32(np.inf)
    rf = float(r)
    if math.isfinite(rf) and rf != 0:
        b = f32_bits(rf) + seed_ulps
        rf = f32_from_bits(b)
    y0 = widen(rf) if math.isfinite(rf) else float("nan")
    if not (-125 <= ex < 126):
        return float("nan")
    e = fma(-x, y0, 1.0)
    return fma(y0, fma(e, e, e), y0)


def ulp(v):
    return math.ulp(abs(v))


def test_seed_is_the_truncated_value_and_the_widening_is_exact():
    rng = np.random.default_rng(1)
    for x in np.exp2(rng.uniform(-124, 125, 2000)) * rng.choice([-1.0, 1.0], 2000):
        x = float(x)
        ex, xf = seed_float(x)
        m, e = math.frexp(x)                       # x = m 2^e, 0.5 <= |m| < 1
        trunc = math.ldexp(math.trunc(m * 2 ** 24) / 2 ** 24, e)
        assert xf == trunc
        assert widen(xf) == xf                     # float32 -> float64 bits, exactly


def test_result_within_one_ulp_of_the_reciprocal():
    rng = np.random.default_rng(2)
    xs = list(np.exp2(rng.uniform(-125, 126, 3000)))
    xs += list(rng.uniform(0.05, 20.0, 3000))      # densities of the workloads
    xs += [1.0, 1.25, 2.0 ** -125, math.nextafter(2.0 ** 126, 0.0), 3.0, 0.1]
    worst = 0.0
    for x in xs:
        x = float(x)
        exact = 1 / Fraction(x)
        for s in (-4, -1, 0, 1, 4):
            y = rcp_nr(x, s)
            err = abs(Fraction(y) - exact) / Fraction(ulp(float(exact)))
            worst = max(worst, float(err))
            assert err <= 1, (x, s, float(err))
        assert rcp_nr(-x, 0) == -rcp_nr(x, 0)
    assert worst > 0.3                             # the bound is not vacuous


def test_out_of_range_inputs_give_nan():
    for x in (0.0, -0.0, 5e-324, 2.0 ** -126, 2.0 ** -1000, 2.0 ** 126, 1e300, math.inf, -math.inf, math.nan):
        assert math.isnan(rcp_nr(x, 0)), x
