"""Planted mistakes: each plausible error in the oracle must fail a pin (CPU only).

The oracle is trusted only because its pins check it against facts that do
not come from its own formulas.  This file shows that the pins would notice:
every case below plants one mistake into the oracle for the duration of the
test (monkeypatch; the oracle's files are not touched) and runs the pins that
should catch it; at least one of them has to fail.  The mistakes are the kind
a restatement of the model gets wrong: a sign, a coefficient, a direction, an
index, a scale factor, a transposed operand.
"""
import numpy as np
import pytest

from oracle import adjoint as A, model as M, observables as O

import test_oracle_adjoint as pa
import test_oracle_bruteforce as pb
import test_oracle_model as pm
import test_oracle_observables as po
import test_oracle_regularized as pr
import test_oracle_transport as pt

K = M.K()
D = M.D
ORIG = {"equilibrium": M.equilibrium, "moments": M.moments, "wall_q": M.wall_q}


# --- planted versions of oracle functions (each differs in one place) -------

def collide_variant(gsign=1.0, tsign=1.0, rate=lambda tau: 1.0 / tau):
    def collide(ft, p):
        out = np.full_like(ft, np.nan)
        fp = M.physical(ft)
        rho, ux, uy, T = M.moments(fp)
        uys = uy - gsign * p.tau * p.g
        Ts = T + tsign * p.tau * (1.0 - p.tau) * p.g * p.g / D
        feq = M.equilibrium(rho, ux, uys, Ts)
        out[:, M.HALO:-M.HALO, :] = fp - (fp - feq) * rate(p.tau)
        return out
    return collide


def equilibrium_cu4_over_12(rho, ux, uy, T):
    """The cu^4 term with 1/12 instead of 1/24."""
    rho, ux, uy, T = np.broadcast_arrays(rho, ux, uy, T)
    extra = np.stack([K["w"][l] * rho * (K["c"][l, 0] * ux + K["c"][l, 1] * uy) ** 4 / 24.0
                      for l in range(M.NPOP)])
    return ORIG["equilibrium"](rho, ux, uy, T) + extra


def equilibrium_theta2_coefficient_2(rho, ux, uy, T):
    """The theta^2 term with 2 instead of 3."""
    rho, ux, uy, T = np.broadcast_arrays(rho, ux, uy, T)
    th = T - 1.0
    c2 = K["c2"]
    extra = np.stack([-K["w"][l] * rho * th * th * (c2[l] ** 2 - 2 * (D + 2) * c2[l] + D * (D + 2)) / 24.0
                      for l in range(M.NPOP)])
    return ORIG["equilibrium"](rho, ux, uy, T) + extra


def moments_wrong_dimension(fp):
    """T from D rho T with D = 3."""
    rho, ux, uy, T = ORIG["moments"](fp)
    return rho, ux, uy, T * D / (D + 1)


def wall_q_scaled(T_wall, wall):
    """q_l off by a common factor, so the unknown slots no longer hold M(x)."""
    return ORIG["wall_q"](T_wall, wall) * 1.001


def propagate_wrong_x_direction(f, p):
    xi = K["xi"]
    ly = p.ly
    out = np.full_like(f, np.nan)
    for l in range(M.NPOP):
        ax, ay = int(xi[l, 0]), int(xi[l, 1])
        if p.periodic_y:
            src = np.roll(f[l, M.HALO:M.HALO + ly, :], ay, axis=0)
        else:
            src = f[l, M.HALO - ay:M.HALO + ly - ay, :]
        out[l, M.HALO:M.HALO + ly, :] = np.roll(src, -ax, axis=1)
    return out


def bc_lost_mass_wrong_column(fprop, fpre, p):
    if p.periodic_y:
        return fprop.copy()
    xi = K["xi"]
    out = fprop.copy()
    ly = p.ly
    for wall, T_wall in (("bottom", p.t_bottom), ("top", p.t_top)):
        q = M.wall_q(T_wall, wall)
        Mx = None
        for (l, y0) in M.lost_terms(wall, ly):
            term = np.roll(fpre[l, M.HALO + y0, :], -int(xi[l, 0]))
            Mx = term.copy() if Mx is None else Mx + term
        for (d, l) in M.unknown_slots(wall):
            y = d if wall == "bottom" else ly - 1 - d
            out[l, M.HALO + y, :] = Mx * q[l]
    return out


def collide_vjp_not_transposed(ft, lam, p):
    fp = M.physical(ft)

    def coll(x):
        full = np.full((M.NPOP,) + ft.shape[1:], np.nan, dtype=x.dtype)
        full[:, M.HALO:-M.HALO] = x
        return M.physical(M.collide(full, p))

    J = A.site_jacobian(coll, fp)
    out = np.full_like(ft, np.nan)
    out[:, M.HALO:-M.HALO] = np.einsum("kl...,l...->k...", J, M.physical(lam))
    return out


def propagate_bc_transpose_wrong_wall_column(mu, p):
    """Pushes each wall cotangent back to the mirrored source column."""
    xi = K["xi"]
    lam = ORIG_T(mu, p)
    if p.periodic_y:
        return lam
    ly = p.ly
    for wall, T_wall in (("bottom", p.t_bottom), ("top", p.t_top)):
        q = M.wall_q(T_wall, wall)
        Lam = 0.0
        for (d, l) in M.unknown_slots(wall):
            y = d if wall == "bottom" else ly - 1 - d
            Lam = Lam + q[l] * mu[l, M.HALO + y, :]
        for (l, y0) in M.lost_terms(wall, ly):
            lam[l, M.HALO + y0, :] = np.roll(Lam, int(xi[l, 0]))
    return lam


ORIG_T = A.propagate_bc_transpose


def observables_fields_wrong_half_impulse(f, p):
    """The mid-step velocity with + g / 2 taken off instead of added."""
    rho, ux, uy, T = M.moments(M.physical(f))
    return rho, ux, uy - 0.5 * p.g, T


def hermite_project_order3_over_3(fp):
    """The order-3 term of the projection divided by 3 instead of 3! = 6."""
    H1, H2, H3, H4 = M._hermite_stack()
    a0 = fp.sum(axis=0)
    a1 = np.einsum("p...,pi->...i", fp, H1)
    a2 = np.einsum("p...,pij->...ij", fp, H2)
    a3 = np.einsum("p...,pijk->...ijk", fp, H3)
    a4 = np.einsum("p...,pijkm->...ijkm", fp, H4)
    out = (a0[None]
           + np.einsum("...i,pi->p...", a1, H1)
           + np.einsum("...ij,pij->p...", a2, H2) / 2.0
           + np.einsum("...ijk,pijk->p...", a3, H3) / 3.0
           + np.einsum("...ijkm,pijkm->p...", a4, H4) / 24.0)
    w = K["w"].reshape((M.NPOP,) + (1,) * (fp.ndim - 1))
    return w * out


def collide_regularized_wrong_factor(ft, p):
    """The projected non-equilibrium part scaled by 1 - tau instead of 1 - 1/tau."""
    out = np.full_like(ft, np.nan)
    fp = M.physical(ft)
    rho, ux, uy, T = M.moments(fp)
    uys = uy - p.tau * p.g
    Ts = T + p.tau * (1.0 - p.tau) * p.g * p.g / D
    feq = M.equilibrium(rho, ux, uys, Ts)
    out[:, M.HALO:-M.HALO, :] = feq + (1.0 - p.tau) * M.hermite_project(fp - feq)
    return out


# --- the pins that should catch each mistake ---------------------------------

def brute():
    pb.test_bruteforce_tiny_lattice_matches_oracle()


def gravity_pin():
    pm.test_collide_gravity_adds_rho_g_and_keeps_rho_and_T()


CASES = [
    ("gravity sign", (M, "collide", collide_variant(gsign=-1.0)), [gravity_pin, brute]),
    ("temperature shift sign", (M, "collide", collide_variant(tsign=-1.0)), [gravity_pin, brute]),
    ("relaxation by tau instead of 1/tau", (M, "collide", collide_variant(rate=lambda tau: tau)),
     [brute, lambda: pt.test_shear_wave_decays_at_the_bgk_viscosity(0.8, 0.7),
      lambda: pt.test_entropy_wave_decays_at_the_bgk_thermal_diffusivity(0.8, 0.7)]),
    ("cu^4 coefficient", (M, "equilibrium", equilibrium_cu4_over_12),
     [pm.test_equilibrium_moments_are_maxwellian_to_order_4, pm.test_equilibrium_closed_form_equals_hermite_tensor_sum,
      brute]),
    ("theta^2 coefficient", (M, "equilibrium", equilibrium_theta2_coefficient_2),
     [pm.test_equilibrium_moments_are_maxwellian_to_order_4, pm.test_equilibrium_closed_form_equals_hermite_tensor_sum,
      brute]),
    ("dimension in eq. (2)", (M, "moments", moments_wrong_dimension), [pm.test_moments_recover_fields, brute]),
    ("wall ratios scaled", (M, "wall_q", wall_q_scaled),
     [pm.test_walls_conserve_mass_exactly_and_ignore_halos, pm.test_walled_lattice_conserves_total_mass_over_steps,
      brute]),
    ("streaming direction in x", (M, "propagate", propagate_wrong_x_direction),
     [lambda: pm.test_propagate_moves_population_along_its_velocity(False),
      lambda: pm.test_propagate_moves_population_along_its_velocity(True), brute]),
    ("lost mass credited to the mirrored column", (M, "bc", bc_lost_mass_wrong_column), [brute]),
    ("collide Jacobian not transposed", (A, "collide_vjp", collide_vjp_not_transposed),
     [pa.test_adjoint_step_dot_product_against_complex_step_jvp]),
    ("wall cotangent pushed to the mirrored column", (A, "propagate_bc_transpose",
                                                      propagate_bc_transpose_wrong_wall_column),
     [lambda: pa.test_propagate_bc_transpose_dot_product(False)]),
    ("mid-step velocity correction sign", (O, "fields", observables_fields_wrong_half_impulse),
     [po.test_free_fall_midpoint_velocity]),
    ("order-3 weight of the Hermite projection", (M, "hermite_project", hermite_project_order3_over_3),
     [pr.test_projection_keeps_moments_to_order_4, pr.test_projection_is_idempotent_and_keeps_equilibrium]),
    ("relaxation factor of the regularised collide", (M, "collide_regularized", collide_regularized_wrong_factor),
     [pr.test_regularized_equals_bgk_inside_the_hermite_space]),
]


@pytest.mark.parametrize("name,patch,pins", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(name, patch, pins, monkeypatch):
    module, attr, planted = patch
    monkeypatch.setattr(module, attr, planted)
    caught = []
    for pin in pins:
        try:
            pin()
        except AssertionError:
            caught.append(pin)
    assert caught, f"no pin caught the planted mistake: {name}"


def test_pins_pass_on_the_oracle_as_it_stands():
    # the same pins, unpatched (so a failure above is the planted mistake's)
    gravity_pin()
    brute()
    pm.test_equilibrium_moments_are_maxwellian_to_order_4()
    pm.test_moments_recover_fields()
    pm.test_walls_conserve_mass_exactly_and_ignore_halos()
    pm.test_propagate_moves_population_along_its_velocity(False)
    pa.test_adjoint_step_dot_product_against_complex_step_jvp()
    pa.test_propagate_bc_transpose_dot_product(False)
    po.test_free_fall_midpoint_velocity()
    pr.test_projection_keeps_moments_to_order_4()
    pr.test_regularized_equals_bgk_inside_the_hermite_space()
