"""Exactness claims of the float64 step's 96-bit fixed-point moment sums,
checked by emulating their word-level steps with Python integers (CPU only).

Each float64 population becomes a 96-bit two's-complement number on the
2^-82 grid (its 53-bit significand shifted by the exponent, split into three
32-bit words), the weighted sums are integer sums modulo 2^96, and the sum is
rounded once to float64 (leading-zero count, funnel shifts, round to nearest
even with a sticky bit).  Checked against rational arithmetic: the result is
the correctly rounded exact sum whenever every population has |f| >= 2^-30
(and |f| < 4), and within one unit in the last place when smaller ones lose
their bits below 2^-82.  Python's int / int division is correctly rounded,
so float(Fraction) is the reference.
"""
import struct
from fractions import Fraction

import numpy as np

M32 = 0xFFFFFFFF
M96 = (1 << 96) - 1
E0 = 993               # biased exponent whose unit in the last place is 2^-82
EMAX = E0 + 31         # |v| < 4


def words(v):
    b = struct.unpack("<Q", struct.pack("<d", v))[0]
    return b >> 32, b & M32


def funnel_l(lo, hi, s):
    """Upper word of (hi:lo) << s, s in 0..31."""
    return ((((hi << 32) | lo) << s) >> 32) & M32


def funnel_r(lo, hi, s):
    """Lower word of (hi:lo) >> s, s in 0..31."""
    return (((hi << 32) | lo) >> s) & M32


def to_fix(v):
    """(96-bit value as an int mod 2^96, ok) following the three-word conversion."""
    hi, lo = words(v)
    e = (hi >> 20) & 0x7FF
    ok = e <= EMAX
    m1 = (hi & 0xFFFFF) | (0x100000 if e != 0 else 0)
    s = e - E0
    if s >= 0:
        t = s & 31
        w0, w1, w2 = (lo << t) & M32, funnel_l(lo, m1, t), funnel_l(m1, 0, t)
    else:
        t = -s
        w0 = funnel_r(lo, m1, t) if t < 32 else (m1 >> (t - 32) if t < 53 else 0)
        w1 = m1 >> t if t < 32 else 0
        w2 = 0
    n = (w2 << 64) | (w1 << 32) | w0
    if hi >> 31:
        n = (-n) & M96
    return n, ok


def clz32(x):
    return 32 - x.bit_length()


def fix_to_double(n):
    w2, w1, w0 = (n >> 64) & M32, (n >> 32) & M32, n & M32
    sign = w2 & 0x80000000
    if sign:
        n = (-n) & M96
        w2, w1, w0 = (n >> 64) & M32, (n >> 32) & M32, n & M32
    if n == 0:
        return 0.0
    n2, n1, n0, lz = w2, w1, w0, 0
    if n2 == 0:
        n2, n1, n0, lz = n1, n0, 0, 32
        if n2 == 0:
            n2, n1, lz = n1, 0, 64
    b = clz32(n2)
    n2, n1, n0 = funnel_l(n1, n2, b), funnel_l(n0, n1, b), (n0 << b) & M32
    lz += b
    m = (n2 << 21) | (n1 >> 11)
    rest = n1 & 0x7FF
    up = rest > 0x400 or (rest == 0x400 and (n0 != 0 or (m & 1)))
    m += 1 if up else 0
    bits = ((13 - lz + 1022) << 52) + m + (sign << 32)
    return struct.unpack("<d", struct.pack("<Q", bits))[0]


def fixed_sum(vals, weights):
    acc = 0
    for k, v in zip(weights, vals):
        n, ok = to_fix(v)
        assert ok
        acc = (acc + k * n) & M96
    return fix_to_double(acc)


def exact_sum(vals, weights):
    return float(sum(k * Fraction(v) for k, v in zip(weights, vals)))


XI = [(0, 0)] + [p for r in [(1, 0), (0, 1), (1, 1), (-1, 1), (2, 0), (0, 2), (2, 1), (1, 2), (-1, 2), (-2, 1),
                              (2, 2), (-2, 2), (3, 0), (0, 3), (3, 1), (1, 3), (-1, 3), (-3, 1)]
                 for p in (r, (-r[0], -r[1]))]
WEIGHTS = [[1] * 37, [x for x, _ in XI], [y for _, y in XI], [x * x + y * y for x, y in XI]]


def populations(rng, tiny=False):
    v = rng.uniform(0.0, 1.0, 37) * 2.0 ** rng.integers(-29, 2, 37)
    v *= np.where(rng.random(37) < 0.2, -1.0, 1.0)
    v[rng.random(37) < 0.05] = 0.0
    if tiny:
        v[rng.integers(0, 37, 4)] = rng.uniform(-1, 1, 4) * 2.0 ** rng.integers(-80, -31, 4)
    return [float(x) for x in v]


def test_conversion_is_exact_down_to_2_to_minus_30():
    rng = np.random.default_rng(0)
    for v in populations(rng) + [3.999999999, -3.5, 2.0 ** -30, -(2.0 ** -30), 1.0, -1.0]:
        n, ok = to_fix(v)
        assert ok
        signed = n - (1 << 96) if n >> 95 else n
        assert Fraction(signed, 1 << 82) == Fraction(v)


def test_out_of_range_values_are_flagged():
    for v in (4.0, -4.0, float("inf"), float("nan"), 1e300):
        assert not to_fix(v)[1]


def test_sums_are_the_correctly_rounded_exact_sums():
    rng = np.random.default_rng(1)
    for _ in range(300):
        vals = populations(rng)
        for w in WEIGHTS:
            assert fixed_sum(vals, w) == exact_sum(vals, w)


def test_rounding_ties_go_to_even_and_carries_reach_the_exponent():
    # 1 + 2^-53 is a tie (rounds to 1), 1 + 3 * 2^-53 rounds up to 1 + 2^-51;
    # 2 - 2^-53 rounds up and carries into the next binade
    cases = [[1.0, 2.0 ** -53], [1.0, 3 * 2.0 ** -53], [2.0, -(2.0 ** -53)], [1.0, 2.0 ** -53, 2.0 ** -60]]
    for vals in cases:
        assert fixed_sum(vals, [1] * len(vals)) == exact_sum(vals, [1] * len(vals))


def test_tiny_populations_stay_within_one_ulp():
    rng = np.random.default_rng(2)
    for _ in range(200):
        vals = populations(rng, tiny=True)
        for w in WEIGHTS:
            got, want = fixed_sum(vals, w), exact_sum(vals, w)
            assert abs(got - want) <= np.spacing(abs(want)), (got, want)
