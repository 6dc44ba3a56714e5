"""Exactness claims of the float32 split moment sums of the FP32-store collide,
checked by emulating its word-level steps in NumPy float32 (CPU only).

NumPy's float32 additions are IEEE round-to-nearest-even, as the device's
add.f32 / sub.f32 are; a fused multiply-add is emulated by forming the exact
result in float64 (the cases below are exact there) and rounding once.  What
is checked, against rational arithmetic:

* the split v = h + m 2^-34 + e with h on the 2^-12 grid, m an integer and
  |e| <= 2^-35, read off as in the kernel ((v + C1) - C1, then the bit
  pattern of (v - h) + C2);
* the weighted sums of the h parts are exact in float32 and the integer sums
  exact modulo 2^32, so a split sum equals the sum of the 2^-34-grid roundings
  exactly;
* the difference of two split sums (the conserved-moment defect of the
  correction pass) is the exact difference rounded once to float32.
"""
from fractions import Fraction

import numpy as np

F = np.float32
C1, C2 = F(3072.0), F(1.5 * 2.0 ** -11)
K2 = int(np.array([C2], dtype=np.float32).view(np.uint32)[0])
XI = np.array([(0, 0)] + [p for r in [(1, 0), (0, 1), (1, 1), (-1, 1), (2, 0), (0, 2), (2, 1), (1, 2), (-1, 2),
                                     (-2, 1), (2, 2), (-2, 2), (3, 0), (0, 3), (3, 1), (1, 3), (-1, 3), (-3, 1)]
                           for p in (r, (-r[0], -r[1]))])


def split(v):
    """h (float32 on the 2^-12 grid) and the 32-bit pattern m + K2."""
    v = np.asarray(v, dtype=F)
    h = (v + C1) - C1
    t = (v - h) + C2
    return h, t.view(np.uint32).astype(np.int64)


def split_sum(d, weights):
    """(h sum in float32, integer sum mod 2^32) of sum_l k_l d_l, k integer."""
    h, bits = split(d)
    hs = F(0.0)
    ms = 0
    for k, hv, b in zip(weights, h, bits):
        if k == 0:
            continue
        hs = F(hs + F(k) * hv)                     # k h: exact (k <= 10, h on a coarse grid)
        ms = (ms + k * (int(b) - K2)) % 2 ** 32
    return hs, ms


def exact_grid_sum(d, weights):
    """sum_l k_l round(d_l, 2^-34) in rationals (round to nearest even)."""
    out = Fraction(0)
    for k, v in zip(weights, d):
        q = Fraction(float(v)) * 2 ** 34
        n = round(q)                               # Python rounds halves to even
        out += k * Fraction(n, 2 ** 34)
    return out


def value(hs, ms):
    m = ms - 2 ** 32 if ms >= 2 ** 31 else ms
    return Fraction(float(hs)) + Fraction(m, 2 ** 34)


def split_diff(b, a):
    """The kernel's difference of two split sums, rounded once to float32."""
    dm = (b[1] - a[1]) % 2 ** 32
    dm = dm - 2 ** 32 if dm >= 2 ** 31 else dm
    dh = F(b[0] - a[0])                            # exact: both on the 2^-12 grid
    inner = F(float(dh) + float(dm >> 12) * 2.0 ** -22)       # exact in float64, exact in float32
    return F(float(inner) + float(dm & 0xFFF) * 2.0 ** -34)   # one rounding


def round_f32(fr):
    """fr rounded to the nearest float32, ties to even, in exact arithmetic."""
    x = F(float(fr))
    cands = [np.nextafter(x, F(-np.inf)), x, np.nextafter(x, F(np.inf))]
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - fr),
                                     int(np.array([c], dtype=F).view(np.uint32)[0]) & 1))
    return best


def deviations(rng, n):
    # float32 deviations d_l = f_l - w_l rho0 of the size the step sees
    scale = rng.choice([1e-1, 1e-2, 1e-3, 1e-5], size=(n, 37))
    return rng.uniform(-1.0, 1.0, size=(n, 37)).astype(F) * scale.astype(F)


WEIGHTS = {
    "rho": np.ones(37, dtype=int),
    "jx": XI[:, 0],
    "jy": XI[:, 1],
    "e": XI[:, 0] ** 2 + XI[:, 1] ** 2,
}


def test_split_parts_reconstruct_each_value_to_the_2_to_34_grid():
    rng = np.random.default_rng(0)
    d = deviations(rng, 50).ravel()
    h, bits = split(d)
    assert np.all(np.asarray(h, dtype=np.float64) * 2 ** 12 == np.round(np.asarray(h, dtype=np.float64) * 2 ** 12))
    for v, hv, b in zip(d, h, bits):
        e = Fraction(float(v)) - Fraction(float(hv)) - Fraction(int(b) - K2, 2 ** 34)
        assert abs(e) <= Fraction(1, 2 ** 35)


def test_split_sums_equal_the_sums_of_grid_rounded_values():
    rng = np.random.default_rng(1)
    for d in deviations(rng, 60):
        for w in WEIGHTS.values():
            assert value(*split_sum(d, w)) == exact_grid_sum(d, w)


def test_difference_of_two_split_sums_is_rounded_once():
    rng = np.random.default_rng(2)
    for d in deviations(rng, 60):
        # a second pass: every population moved a little (the relaxation),
        # the sums nearly unchanged (the defect is tiny)
        d2 = (d + rng.uniform(-1e-3, 1e-3, size=37).astype(F)).astype(F)
        for w in WEIGHTS.values():
            a, b = split_sum(d, w), split_sum(d2, w)
            exact = value(*b) - value(*a)
            assert split_diff(b, a) == round_f32(exact)
