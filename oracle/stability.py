"""Linear stability of the plain BGK D2Q37 step about a fluid at rest
(oracle side; test infrastructure).

The paper states the model and its kernels (Sect. 2) but no stability range;
it only mentions a projection onto Hermite polynomials "for stability".  The
readings of ``oracle.model`` (4th-order Hermite equilibrium about T0 = 1,
plain BGK, eq. (1)) fix where a uniform fluid is stable, and this module
computes it from the oracle itself:

* f* = f^eq(rho, 0, T) is a fixed point of one step on a periodic lattice
  with g = 0 (propagate moves a uniform state onto itself, collide keeps an
  equilibrium);
* a Fourier perturbation df_l(x) = a_l exp(i k.x) evolves as a -> J S(k) a,
  with J the 37 x 37 Jacobian of ``oracle.model.collide`` at f* (complex
  step, as in ``oracle.adjoint``) and S(k) = diag(exp(-i k.xi_l)) the symbol
  of the pull propagate f_l(x) <- f_l(x - xi_l);
* the state is linearly unstable when the spectral radius of J S(k) exceeds
  one for some k.  The square symmetry of the velocity set makes k in
  [0, pi]^2 enough.

Run as a script to print the (T, tau) table.
"""
from __future__ import annotations

import numpy as np

from . import adjoint as A, lattice, model as M


def collide_jacobian(T, tau, rho=1.0):
    """37 x 37 Jacobian of collide at the rest equilibrium f^eq(rho, 0, T), g = 0."""
    p = M.Params(1, 1, tau=tau, g=0.0, periodic_y=True)
    fstar = M.equilibrium(np.array([[rho]]), np.zeros((1, 1)), np.zeros((1, 1)), np.array([[T]]))

    def coll(x):
        full = np.full((M.NPOP, 1 + 2 * M.HALO, 1), np.nan, dtype=x.dtype)
        full[:, M.HALO:-M.HALO] = x
        return M.physical(M.collide(full, p))

    return A.site_jacobian(coll, fstar)[:, :, 0, 0]


def shift_symbol(kx, ky):
    """diag(exp(-i k.xi_l)) of the pull propagate."""
    xi = lattice.constants()["xi"]
    return np.exp(-1j * (kx * xi[:, 0] + ky * xi[:, 1]))


def max_growth(T, tau, nk=33, rho=1.0):
    """max over k in [0, pi]^2 (nk x nk grid) of the spectral radius of
    J S(k); returns (radius, kx, ky)."""
    J = collide_jacobian(T, tau, rho)
    best = (0.0, 0.0, 0.0)
    for kx in np.linspace(0.0, np.pi, nk):
        for ky in np.linspace(0.0, np.pi, nk):
            r = np.abs(np.linalg.eigvals(J * shift_symbol(kx, ky)[None, :])).max()
            if r > best[0]:
                best = (float(r), float(kx), float(ky))
    return best


def min_equilibrium_population(T, rho=1.0):
    """min over l of f^eq_l(rho, 0, T) / (w_l rho): negative where the
    4th-order equilibrium turns negative on some shell."""
    w = lattice.constants()["w"]
    f = M.equilibrium(np.array([rho]), np.zeros(1), np.zeros(1), np.array([T]))[:, 0]
    q = f / (w * rho)
    return float(q.min()), int(np.argmin(q))


def first_nonfinite_step(f, p: M.Params, max_steps: int, every: int = 10):
    """Step the oracle and return the first multiple of `every` after which
    a physical population is not finite (None if all stay finite)."""
    for i in range(1, max_steps + 1):
        f = M.step(f, p)
        if i % every == 0 and not np.isfinite(M.physical(f)).all():
            return i
    return None


def table(Ts=(0.5, 0.6, 0.7, 0.75, 1.0, 1.25, 1.5), taus=(0.55, 0.6, 0.7, 0.8, 1.0), nk=33):
    return {(T, tau): max_growth(T, tau, nk)[0] for T in Ts for tau in taus}


def rt_slab_divergence(width=64, lx=2048, ly=4096, max_steps=400):
    """First non-finite step of the oracle on a `width`-column slab (periodic
    in x) of the 2048 x 4096 Rayleigh-Taylor workload: T = 0.5 / 1.5, 32
    modes, seed 0, tau = 0.6, g = 1e-5."""
    import synth
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 32, 0)
    p = M.Params(width, ly, tau=0.6, g=1e-5, t_top=tt, t_bottom=tb)
    f = M.init_state(rho[:, :width], ux[:, :width], uy[:, :width], T[:, :width])
    return first_nonfinite_step(f, p, max_steps)


if __name__ == "__main__":
    import sys
    if len(sys.argv) > 1 and sys.argv[1] == "rt-slab":
        print("first non-finite step, 64-column slab of the 2048 x 4096 RT workload:", rt_slab_divergence())
        sys.exit(0)
    Ts = (0.5, 0.6, 0.7, 0.75, 1.0, 1.25, 1.5)
    taus = (0.55, 0.6, 0.7, 0.8, 1.0)
    print("max spectral radius of J S(k), k in [0, pi]^2 (33 x 33 grid); > 1 is unstable")
    print("T \\ tau " + " ".join(f"{t:>10}" for t in taus))
    for T in Ts:
        print(f"{T:7} " + " ".join(f"{max_growth(T, tau)[0]:10.6f}" for tau in taus))
    for T in Ts:
        q, l = min_equilibrium_population(T)
        print(f"T = {T}: min_l f^eq_l / (w_l rho) = {q:.4f} (population {l})")
