"""The float64 step's folded equilibrium coefficients (eq_monomials_moments in
lbm_device.cuh), restated in Python float64 step by step and checked against
the oracle's closed-form equilibrium with the gravity shift (CPU only).

The kernel never forms u or T: from the moment sums rho, J and E / 2 (integer
velocities xi, c = r xi) it takes s = r^2 / rho, the shifted velocity
v = (J_x s, J_y s - r^2 tau g / r), U2 = |v|^2 / r^2 and
theta = (E / 2) s - U2 / 2 - (tau g / r) v_y + tshift - (r^2 / 2) (tau g / r)^2,
folds the Hermite coefficients (B10 = 2 (h - theta), B01 r^2 = (theta r^2 / 2)
B10, 1 - U2 / 2 + U2^2 / 8 = 2 h^2 + 1/2, theta^2 r^4 / 8 = (theta r^2 / 2)
(theta r^2 / 4)) and halves the xy coefficient (doubled exactly in fixed
point).  Here the same operations run in Python float64 (FMAs through exact
rationals), the polynomial is summed exactly, and w_l rho P(xi_l) must match
the oracle's equilibrium(rho, u_x, u_y - tau g, T + tau (1 - tau) g^2 / 2)
within 1e-13 of each population's size.  A dropped gravity term, a wrong
half or a wrong sign in any fold moves some population by far more.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import lattice, model as M

K = lattice.constants()
R = float(K["r"])
R2 = R * R
XI = K["xi"].astype(int)
# monomial exponents (c, e) of xi_x^c xi_y^e in the kernel's order
MONO = [(0, 0), (2, 0), (0, 2), (4, 0), (2, 2), (0, 4), (1, 0), (3, 0), (1, 2),
        (0, 1), (0, 3), (2, 1), (1, 1), (3, 1), (1, 3)]


def fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def folded_coefficients(rho, Jx, Jy, Eh, tau, g):
    tau_g_xi = tau * g / R
    tshift = tau * (1.0 - tau) * g * g / 2.0 - 1.0
    r2_2, r2_4 = 0.5 * R2, 0.25 * R2
    tshift_v = tshift - r2_2 * tau_g_xi * tau_g_xi
    inv_r2 = 1.0 / R2
    s = R2 * (1.0 / rho)
    vx = Jx * s
    vy = fma(Jy, s, -(R2 * tau_g_xi))
    vx2, vy2, vxy = vx * vx, vy * vy, vx * vy
    v2 = vx2 + vy2
    U2 = v2 * inv_r2
    theta = fma(Eh, s, fma(-0.5, U2, fma(-tau_g_xi, vy, tshift_v)))
    h, h2 = fma(-0.25, U2, 0.5), fma(-0.5, U2, 1.0)
    B20 = fma(-1.5, theta, h)
    B10 = fma(-2.0, theta, h2)
    B00 = fma(theta, (U2 - 1.0) + theta, fma(h2, h, 0.5))
    t4, t2 = theta * r2_4, theta * r2_2
    B01r2 = t2 * B10
    q8, q4 = t2 * t4, t2 * t2
    I, J = fma(vx2, 1.0 / 6.0, t2), fma(vy2, 1.0 / 6.0, t2)
    P = [B00, fma(B20, vx2, B01r2), fma(B20, vy2, B01r2),
         fma(vx2, fma(vx2, 1.0 / 24.0, t4), q8), fma(t4, v2, fma(0.25 * vxy, vxy, q4)),
         fma(vy2, fma(vy2, 1.0 / 24.0, t4), q8),
         B10 * vx, vx * I, vx * fma(0.5, vy2, t2), B10 * vy, vy * J, vy * fma(0.5, vx2, t2),
         B20 * vxy, vxy * I, vxy * J]
    P[12] = 2 * P[12]          # the half is doubled exactly (fixed point)
    return P


def test_folded_coefficients_reproduce_the_shifted_equilibrium():
    lx, ly = 6, 5
    rng = np.random.default_rng(7)
    worst = 0.0
    for trial in range(4):
        rho, ux, uy, T = synth.random_fields(lx, ly, 30 + trial, umax=0.1)
        tau, g = float(rng.uniform(0.55, 1.2)), float(rng.uniform(0.0, 3e-3))
        f = M.init_state(rho, ux, uy, T)[:, 3:-3]
        f = f * (1.0 + 0.02 * synth.noise(lx, ly, 40 + trial))
        r_o, ux_o, uy_o, T_o = M.moments(f)
        feq = M.equilibrium(r_o, ux_o, uy_o - tau * g, T_o + tau * (1.0 - tau) * g * g / 2.0)
        for y in range(ly):
            for x in range(lx):
                col = [Fraction(v) for v in f[:, y, x]]
                rho_s = float(sum(col))
                Jx = float(sum(v * int(c[0]) for v, c in zip(col, XI)))
                Jy = float(sum(v * int(c[1]) for v, c in zip(col, XI)))
                Eh = float(sum(v * int(c[0] ** 2 + c[1] ** 2) for v, c in zip(col, XI)) / 2)
                P = folded_coefficients(rho_s, Jx, Jy, Eh, tau, g)
                for l in range(37):
                    a, b = int(XI[l, 0]), int(XI[l, 1])
                    val = sum(Fraction(P[m]) * a ** c * b ** e for m, (c, e) in enumerate(MONO))
                    got = float(Fraction(K["w"][l]) * Fraction(rho_s) * val)
                    want = feq[l, y, x]
                    err = abs(got - want) / abs(want)
                    worst = max(worst, err)
                    assert err <= 1e-13, (trial, l, err)
    assert worst > 1e-17                          # the comparison is not vacuous


@pytest.mark.parametrize("mistake", ["gravity", "half", "coefficient_sign"])
def test_a_planted_mistake_in_the_folds_is_caught(mistake, monkeypatch):
    # the same check with one fold broken must fail
    orig = folded_coefficients

    def broken(rho, Jx, Jy, Eh, tau, g):
        if mistake == "gravity":
            return orig(rho, Jx, Jy, Eh, tau, 0.0 if g else g)
        P = orig(rho, Jx, Jy, Eh, tau, g)
        if mistake == "half":
            P[12] = P[12] / 2
        else:
            P[1], P[2] = -P[1], -P[2]
        return P

    monkeypatch.setitem(globals(), "folded_coefficients", broken)
    with pytest.raises(AssertionError):
        test_folded_coefficients_reproduce_the_shifted_equilibrium()
