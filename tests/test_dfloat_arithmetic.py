"""Error bounds of the double-float ("double-word") building blocks used by
the FP64_DF collide, the FP32-store collide and the double-float adjoint,
checked by emulating each algorithm word by word in NumPy float32 (CPU only).

float32 additions, subtractions and products are NumPy's (IEEE round to
nearest even, as the device's); a fused multiply-add is the exact rational
result rounded once.  The bounds are those published for the algorithms
(Joldes, Muller and Popescu, ACM TOMS 44, 2017), u = 2^-24:

* TwoSum, Fast2Sum (|a| >= |b|) and the FMA TwoProd are error-free;
* DWPlusFP: relative error <= 2 u^2;
* AccurateDWPlusDW: <= 3 u^2 + 13 u^3;
* SloppyDWPlusDW: <= 3 u^2 relative to |x| + |y| (it is used only where the
  sum does not cancel);
* DWTimesFP (FMA variant): <= 2 u^2;
* DWTimesDW (FMA variant): <= 5 u^2;
* the reciprocal (float seed, one double-word Newton step): measured
  <= 2.9 u^2, tested against 4 u^2;
* the float64 -> double-word conversion by bit arithmetic: <= 2^-48 |x| for
  |x| >= 2^-74, <= 2^-24 |x| below (the low word would be subnormal), 0 below
  2^-126, NaN from 2^128 on; and float32 -> float64 by bit arithmetic is exact.
"""
import struct
from fractions import Fraction

import numpy as np
import pytest

F = np.float32
U = Fraction(1, 2 ** 24)
N = 1500


def bits32(x):
    return int(np.array([x], dtype=F).view(np.uint32)[0])


def f32_from_bits(i):
    return F(struct.unpack("<f", struct.pack("<I", i & 0xFFFFFFFF))[0])


def rn32(fr):
    """fr rounded to the nearest float32, ties to even (exact)."""
    x = F(float(fr))
    cands = [np.nextafter(x, F(-np.inf)), x, np.nextafter(x, F(np.inf))]
    return min(cands, key=lambda c: (abs(Fraction(float(c)) - fr), bits32(c) & 1))


def fma(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def fast_two_sum(a, b):
    s = F(a + b)
    return s, F(b - F(s - a))


def two_prod(a, b):
    p = F(a * b)
    return p, fma(a, b, -p)


def dw_plus_fp(x, y):
    sh, sl = two_sum(x[0], y)
    return fast_two_sum(sh, F(x[1] + sl))


def sloppy_dw_plus_dw(x, y):
    sh, sl = two_sum(x[0], y[0])
    return fast_two_sum(sh, F(sl + F(x[1] + y[1])))


def accurate_dw_plus_dw(x, y):
    sh, sl = two_sum(x[0], y[0])
    th, tl = two_sum(x[1], y[1])
    vh, vl = fast_two_sum(sh, F(sl + th))
    return fast_two_sum(vh, F(tl + vl))


def dw_times_fp(x, y):
    ch, cl = two_prod(x[0], y)
    return fast_two_sum(ch, fma(x[1], y, cl))


def dw_times_dw(x, y):
    ch, cl = two_prod(x[0], y[0])
    t = fma(x[0], y[1], F(x[1] * y[0]))
    return fast_two_sum(ch, F(cl + t))


def dw_rcp(x):
    r = F(F(1.0) / x[0])
    xr = dw_times_fp(x, r)
    e = dw_plus_fp((-xr[0], -xr[1]), F(1.0))
    return dw_plus_fp(dw_times_fp(e, r), r)


def val(x):
    return Fraction(float(x[0])) + Fraction(float(x[1]))


def rand_fp(rng):
    return F(rng.uniform(0.5, 2.0) * (1 if rng.random() < 0.5 else -1) * 2.0 ** int(rng.integers(-12, 12)))


def rand_dw(rng):
    h = rand_fp(rng)
    return fast_two_sum(h, F(float(h) * 2.0 ** -24 * rng.uniform(-0.5, 0.5)))


def rel(got, want):
    return abs(got - want) / abs(want)


def test_error_free_transforms_are_exact():
    rng = np.random.default_rng(0)
    for _ in range(N):
        a, b = rand_fp(rng), rand_fp(rng)
        assert val(two_sum(a, b)) == Fraction(float(a)) + Fraction(float(b))
        big, small = (a, b) if abs(a) >= abs(b) else (b, a)
        assert val(fast_two_sum(big, small)) == Fraction(float(a)) + Fraction(float(b))
        assert val(two_prod(a, b)) == Fraction(float(a)) * Fraction(float(b))


@pytest.mark.parametrize("name,op,bound,kind", [
    ("DWPlusFP", dw_plus_fp, 2 * U ** 2, "fp"),
    ("AccurateDWPlusDW", accurate_dw_plus_dw, 3 * U ** 2 + 13 * U ** 3, "dw"),
    ("DWTimesFP", dw_times_fp, 2 * U ** 2, "fp"),
    ("DWTimesDW", dw_times_dw, 5 * U ** 2, "dw"),
])
def test_double_word_operations_meet_their_bounds(name, op, bound, kind):
    rng = np.random.default_rng(1)
    is_sum = "Plus" in name
    for _ in range(N):
        x = rand_dw(rng)
        y = rand_fp(rng) if kind == "fp" else rand_dw(rng)
        vy = Fraction(float(y)) if kind == "fp" else val(y)
        want = val(x) + vy if is_sum else val(x) * vy
        if want == 0:
            continue
        assert rel(val(op(x, y)), want) <= bound, name


def test_sloppy_sum_error_is_bounded_by_the_operand_magnitudes():
    rng = np.random.default_rng(2)
    for _ in range(N):
        x, y = rand_dw(rng), rand_dw(rng)
        err = abs(val(sloppy_dw_plus_dw(x, y)) - (val(x) + val(y)))
        assert err <= 3 * U ** 2 * (abs(val(x)) + abs(val(y)))


def test_reciprocal_is_accurate_to_a_few_u_squared():
    rng = np.random.default_rng(3)
    for _ in range(N):
        x = rand_dw(rng)
        assert rel(val(dw_rcp(x)), 1 / val(x)) <= 4 * U ** 2


def from_double_bits(x):
    """The float64 -> double-word conversion by integer arithmetic on the bits."""
    b = struct.unpack("<Q", struct.pack("<d", x))[0]
    mag = b & 0x7FFFFFFFFFFFFFFF
    sign = (b >> 32) & 0x80000000
    e = mag >> 52
    H = (mag + (1 << 28)) & ~((1 << 29) - 1)
    hbits = (H >> 29) - (896 << 23)
    D = mag - H
    scale = f32_from_bits(max(e - 948, 1) << 23)
    lo = F(F(D) * scale)
    hi = f32_from_bits(hbits) if 0 <= hbits < 2 ** 32 else F(0)
    if e < 897:
        hi, lo = F(0), F(0)
    if e > 1150:
        hi, lo = F(np.nan), F(0)
    if e < 949:
        lo = F(0)
    return f32_from_bits(bits32(hi) | sign), f32_from_bits(bits32(lo) ^ sign)


def test_float64_to_double_word_by_bits():
    rng = np.random.default_rng(4)
    for lo_e, hi_e, bound in ((-73, 127, Fraction(1, 2 ** 48)), (-125, -75, Fraction(1, 2 ** 24))):
        for _ in range(N):
            x = float(rng.uniform(0.5, 1.0) * (1 if rng.random() < 0.5 else -1) * 2.0 ** int(rng.integers(lo_e, hi_e)))
            assert rel(val(from_double_bits(x)), Fraction(x)) <= bound
    assert val(from_double_bits(1e-40)) == 0
    assert np.isnan(from_double_bits(2.0 ** 128)[0]) and np.isnan(from_double_bits(float("inf"))[0])
    h, l = from_double_bits(-1.5)
    assert (h, l) == (F(-1.5), F(0.0)) and bits32(l) == 0x80000000


def f32_to_f64_bits(v):
    u = bits32(v)
    e = (u >> 23) & 0xFF
    sign = (u & 0x80000000) << 32
    m = (u & 0x7FFFFF) << 29
    ex = 0x7FF if e == 255 else e + 896
    b = sign if e == 0 else (sign | (ex << 52) | m)
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def test_float32_to_float64_by_bits_is_exact_for_normal_floats():
    rng = np.random.default_rng(5)
    for _ in range(N):
        v = F(rng.uniform(0.5, 1.0) * (1 if rng.random() < 0.5 else -1) * 2.0 ** int(rng.integers(-125, 127)))
        assert f32_to_f64_bits(v) == float(v)
    assert np.isinf(f32_to_f64_bits(F(np.inf))) and np.isnan(f32_to_f64_bits(F(np.nan)))
    assert f32_to_f64_bits(F(5e-39)) == 0.0        # subnormals give 0, as documented
