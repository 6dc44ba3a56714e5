"""D2Q37 velocity set and quadrature weights (oracle side; test infrastructure).

The paper uses a D2Q37 model with 37 populations that hop up to three sites
per step (Sect. 2, Fig. "streamscheme" and the propagate bullet) and that
enforces the perfect-gas law p = rho T; it leaves the velocity set and the
weights to the works it cites.  The reading taken here:

* Integer velocities xi with |xi_x|, |xi_y| <= 3 and |xi|^2 in
  {0, 1, 2, 4, 5, 8, 9, 10}: 1 + 4 + 4 + 4 + 8 + 4 + 4 + 8 = 37.
* Lattice velocities c_l = r * xi_l with one scale r.
* Weights w_s per shell and r chosen so that every even moment of order
  <= 8 of the discrete set equals that of a unit-variance Gaussian:
  sum_l w_l c_lx^a c_ly^b = (a-1)!! (b-1)!!  for a, b even, a + b <= 8
  (odd moments vanish by symmetry).  With the square symmetry these are nine
  independent equations for nine unknowns (eight weights and r).

Population order (part of the library interface): l = 0 is the rest
population; for k = 0..17, l = 2k+1 is +xi_k and l = 2k+2 is -xi_k, with the
representatives xi_k listed in ``PAIR_REPS``.

The system is solved exactly: for y = 1/r^2 the equations are linear in the
weights with integer coefficients, so the solvability condition
det[M | rhs(y)] = 0 is a quartic in y with rational coefficients, computed
here with ``fractions.Fraction``; its root and the weights are then found in
``decimal`` arithmetic at 60 digits and rounded once to float64.
"""
from __future__ import annotations

from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np

D = 2
NPOP = 37
SHELLS = (0, 1, 2, 4, 5, 8, 9, 10)

# Representatives +xi_k of the 18 (+xi, -xi) pairs, by shell.
PAIR_REPS = (
    (1, 0), (0, 1),                    # |xi|^2 = 1
    (1, 1), (-1, 1),                   # 2
    (2, 0), (0, 2),                    # 4
    (2, 1), (1, 2), (-1, 2), (-2, 1),  # 5
    (2, 2), (-2, 2),                   # 8
    (3, 0), (0, 3),                    # 9
    (3, 1), (1, 3), (-1, 3), (-3, 1),  # 10
)


def velocities():
    """The 37 integer velocities xi_l in library order, as a (37, 2) int array."""
    v = [(0, 0)]
    for (a, b) in PAIR_REPS:
        v.append((a, b))
        v.append((-a, -b))
    return np.array(v, dtype=np.int64)


def _shell_members(s):
    return [(a, b) for a in range(-3, 4) for b in range(-3, 4) if a * a + b * b == s]


# Monomials xi_x^a xi_y^b (a >= b, both even) whose sums give the nine
# independent isotropy conditions, with the Gaussian moment (a-1)!!(b-1)!!.
_MONOMIALS = ((0, 0), (2, 0), (4, 0), (2, 2), (6, 0), (4, 2), (8, 0), (6, 2), (4, 4))


def _dfact(n):
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def _gauss(a, b):
    return _dfact(a - 1) * _dfact(b - 1)


def _moment_matrix():
    """Integer matrix A[i][s] = sum over shell s of xi_x^a xi_y^b for monomial i."""
    return [[sum(x ** a * y ** b for (x, y) in _shell_members(s)) for s in SHELLS]
            for (a, b) in _MONOMIALS]


def _det(m):
    """Exact determinant of a square matrix of Fractions (Gaussian elimination)."""
    m = [[Fraction(v) for v in row] for row in m]
    n = len(m)
    det = Fraction(1)
    for c in range(n):
        p = next((r for r in range(c, n) if m[r][c] != 0), None)
        if p is None:
            return Fraction(0)
        if p != c:
            m[c], m[p] = m[p], m[c]
            det = -det
        det *= m[c][c]
        for r in range(c + 1, n):
            f = m[r][c] / m[c][c]
            if f:
                for k in range(c, n):
                    m[r][k] -= f * m[c][k]
    return det


def solvability_quartic():
    """Coefficients p[0..4] (Fractions) of det[A | rhs(y)] = sum_k p[k] y^k.

    Row i of rhs(y) is (a_i-1)!!(b_i-1)!! y^((a_i+b_i)/2), y = 1/r^2.  The
    determinant is expanded along that last column.
    """
    A = _moment_matrix()
    n = len(A)  # 9 rows, 8 columns
    p = [Fraction(0)] * 5
    for i, (a, b) in enumerate(_MONOMIALS):
        minor = [row for r, row in enumerate(A) if r != i]
        cof = (-1) ** (i + n - 1) * _det(minor)
        p[(a + b) // 2] += _gauss(a, b) * cof
    return p


def _solve_linear_dec(A, rhs):
    """Solve the square system A w = rhs in Decimal (partial pivoting)."""
    n = len(A)
    m = [[Decimal(v) for v in A[r]] + [rhs[r]] for r in range(n)]
    for c in range(n):
        p = max(range(c, n), key=lambda r: abs(m[r][c]))
        m[c], m[p] = m[p], m[c]
        for r in range(n):
            if r != c and m[r][c] != 0:
                f = m[r][c] / m[c][c]
                for k in range(c, n + 1):
                    m[r][k] -= f * m[c][k]
    return [m[r][n] / m[r][r] for r in range(n)]


def solve_quadrature(digits: int = 60):
    """Return (r, weights_by_shell) as Decimals, weights keyed by |xi|^2.

    The root y of the quartic is bracketed on (0.5, 1) and refined by
    bisection; the weights follow from eight of the equations; all nine
    residuals are checked.
    """
    getcontext().prec = digits
    p = [Decimal(q.numerator) / Decimal(q.denominator) for q in solvability_quartic()]

    def poly(y):
        return (((p[4] * y + p[3]) * y + p[2]) * y + p[1]) * y + p[0]

    lo, hi = Decimal("0.5"), Decimal("1.0")
    flo = poly(lo)
    if flo * poly(hi) > 0:
        raise RuntimeError("quadrature root not bracketed")
    for _ in range(digits * 4):
        mid = (lo + hi) / 2
        fm = poly(mid)
        if fm == 0:
            lo = hi = mid
            break
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    y = (lo + hi) / 2
    A = _moment_matrix()
    rhs = [Decimal(_gauss(a, b)) * y ** ((a + b) // 2) for (a, b) in _MONOMIALS]
    # Drop the equation whose complementary 8x8 minor is largest (some 8x8
    # subsets are singular), solve the other eight, check all nine.
    drop = max(range(9), key=lambda i: abs(_det([row for k, row in enumerate(A) if k != i])))
    keep = [i for i in range(9) if i != drop]
    w = _solve_linear_dec([A[i] for i in keep], [rhs[i] for i in keep])
    res = max(abs(sum(Decimal(A[i][s]) * w[s] for s in range(8)) - rhs[i]) for i in range(9))
    if res > Decimal(10) ** (-(digits - 15)):
        raise RuntimeError(f"quadrature residual too large: {res}")
    if any(v <= 0 for v in w):
        raise RuntimeError("non-positive quadrature weight")
    r = 1 / y.sqrt()
    return r, dict(zip(SHELLS, w)), y


_CACHE = {}


def constants():
    """Float64 constants: dict with r, xi (37x2 int), c (37x2), w (37,), c2 (37,).

    r and the weights are the float64 values nearest to the exact solution;
    c_l = r xi_l and |c_l|^2 = r^2 |xi_l|^2 are rounded once from 60-digit
    values.
    """
    if "c" in _CACHE:
        return _CACHE["c"]
    r, ws, y = solve_quadrature()
    xi = velocities()
    shell = (xi ** 2).sum(axis=1)
    w = np.array([float(ws[int(s)]) for s in shell])
    c = np.array([[float(r * int(a)), float(r * int(b))] for a, b in xi])
    c2 = np.array([float(int(s) / y) for s in shell])
    out = dict(r=float(r), r_dec=r, y_dec=y, w_dec=ws, xi=xi, shell=shell, w=w, c=c, c2=c2)
    _CACHE["c"] = out
    return out
