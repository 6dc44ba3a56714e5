"""Pins of the oracle's D2Q37 velocity set and quadrature (CPU only).

The paper names the D2Q37 model (Sect. 2) but defers its definition; these
tests pin the oracle's reconstruction against facts fixed by mathematics:
Gaussian moments, symmetry, and published values of the D2V37 quadrature.
"""
import math
import os

import numpy as np
import pytest

from oracle import lattice

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def gauss1(k):
    """k-th moment of a unit normal variable."""
    if k % 2:
        return 0.0
    return float(math.prod(range(k - 1, 0, -2))) if k > 0 else 1.0


def test_velocity_set_structure():
    xi = lattice.velocities()
    assert xi.shape == (37, 2)
    assert len({tuple(v) for v in xi}) == 37
    assert tuple(xi[0]) == (0, 0)
    for k in range(18):
        assert tuple(xi[2 * k + 1]) == tuple(-xi[2 * k + 2])
    assert np.abs(xi).max() == 3              # hops of up to three sites (Sect. 2)
    shells = sorted((xi ** 2).sum(1).tolist())
    counts = {s: shells.count(s) for s in set(shells)}
    assert counts == {0: 1, 1: 4, 2: 4, 4: 4, 5: 8, 8: 4, 9: 4, 10: 8}


def test_quadrature_matches_gaussian_moments_to_order_9():
    k = lattice.constants()
    w, c = k["w"], k["c"]
    assert abs(w.sum() - 1.0) < 1e-15
    for a in range(10):
        for b in range(10 - a):
            got = float((w * c[:, 0] ** a * c[:, 1] ** b).sum())
            want = gauss1(a) * gauss1(b)
            assert abs(got - want) <= 2e-14 * max(1.0, abs(want)), (a, b, got, want)


def test_quadrature_is_not_exact_at_order_10():
    # The set is exactly an order-9 rule: a degree-10 moment must differ.
    k = lattice.constants()
    got = float((k["w"] * k["c"][:, 0] ** 10).sum())
    assert abs(got - gauss1(10)) > 1.0


def test_quadrature_literature_values():
    # D2V37 lattice of Philippi, Hegele, dos Santos and Surmas, Phys. Rev. E 73,
    # 056702 (2006), the velocity set of the thermal D2Q37 model the paper cites
    # for its physics (Sect. 2, refs. JFM and POF).  Values as published.
    ref = {}
    with open(os.path.join(GOLDEN, "d2v37_literature.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                key, val = line.split()
                ref[key] = float(val)
    k = lattice.constants()
    assert k["r"] == pytest.approx(ref["r"], rel=1e-15)
    shell_w = {int(s): float(v) for s, v in k["w_dec"].items()}
    for s in (0, 1, 2, 4, 5, 8, 9, 10):
        assert shell_w[s] == pytest.approx(ref[f"w{s}"], rel=1e-14), s


def test_quadrature_golden_regression():
    # Written by tests/golden/make_golden.py from the oracle's 60-digit solve.
    k = lattice.constants()
    vals = {}
    with open(os.path.join(GOLDEN, "d2q37_constants.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                key, val = line.split()
                vals[key] = float.fromhex(val)
    assert k["r"] == vals["r"]
    for l in range(37):
        assert k["w"][l] == vals[f"w_{l}"]
