"""Brute-force pin: a per-site, per-population loop restatement of one D2Q37
step on a tiny lattice, compared with the vectorised oracle (CPU only).

The loop version is written from the model's statement directly: streaming by
following each population along its velocity, the wall mass balance by
collecting what crosses each wall, eq. (2) by explicit sums, and the
equilibrium by the explicit Hermite-tensor series.  It shares only the
velocity set and weights with the oracle (pinned in test_oracle_lattice).
"""
import numpy as np

import synth
from oracle import lattice, model as M

K = lattice.constants()
XI = K["xi"]
C = K["c"]
W = K["w"]
H = [M._hermite_tensors(C[l]) for l in range(37)]


def feq_site(rho, u, T):
    th = T - 1.0
    I = np.eye(2)
    uu = np.outer(u, u)
    a2 = uu + th * I
    a3 = np.einsum("i,j,k->ijk", u, u, u) + th * (
        np.einsum("i,jk->ijk", u, I) + np.einsum("j,ik->ijk", u, I) + np.einsum("k,ij->ijk", u, I))
    s6 = sum(np.einsum(e, uu, I) for e in ("ij,kl->ijkl", "ik,jl->ijkl", "il,jk->ijkl",
                                             "jk,il->ijkl", "jl,ik->ijkl", "kl,ij->ijkl"))
    s3 = sum(np.einsum(e, I, I) for e in ("ij,kl->ijkl", "ik,jl->ijkl", "il,jk->ijkl"))
    a4 = np.einsum("i,j,k,l->ijkl", u, u, u, u) + th * s6 + th * th * s3
    out = np.empty(37)
    for l in range(37):
        H1, H2, H3, H4 = H[l]
        out[l] = W[l] * rho * (1 + u @ H1 + (a2 * H2).sum() / 2 + (a3 * H3).sum() / 6
                               + (a4 * H4).sum() / 24)
    return out


def brute_step(f, lx, ly, tau, g, t_top, t_bottom):
    ft = np.full((37, ly, lx), np.nan)
    lost = {"bottom": np.zeros(lx), "top": np.zeros(lx)}
    # streaming: follow every population from its site along its velocity
    for y in range(ly):
        for x in range(lx):
            for l in range(37):
                tx = (x + XI[l, 0]) % lx
                ty = y + XI[l, 1]
                v = f[l, y + 3, x]
                if ty < 0:
                    lost["bottom"][tx] += v
                elif ty >= ly:
                    lost["top"][tx] += v
                else:
                    ft[l, ty, tx] = v
    # walls: unfilled slots share the lost mass of their column as f^eq(1, 0, T_wall)
    for wall, Tw in (("bottom", t_bottom), ("top", t_top)):
        phi = feq_site(1.0, np.zeros(2), Tw)
        rows = range(0, 3) if wall == "bottom" else range(ly - 3, ly)
        for x in range(lx):
            slots = [(y, l) for y in rows for l in range(37) if np.isnan(ft[l, y, x])
                     and not (0 <= y - XI[l, 1] < ly)]
            tot = sum(phi[l] for (_, l) in slots)
            for (y, l) in slots:
                ft[l, y, x] = lost[wall][x] * phi[l] / tot
    assert np.isfinite(ft).all()
    out = np.full_like(f, np.nan)
    for y in range(ly):
        for x in range(lx):
            fs = ft[:, y, x]
            rho = sum(fs[l] for l in range(37))
            u = sum(C[l] * fs[l] for l in range(37)) / rho
            T = sum(((C[l] - u) ** 2).sum() * fs[l] for l in range(37)) / (2 * rho)
            us = u + tau * np.array([0.0, -g])
            Ts = T + tau * (1 - tau) * g * g / 2
            fe = feq_site(rho, us, Ts)
            out[:, y + 3, x] = fs - (fs - fe) / tau
    return out


def test_bruteforce_tiny_lattice_matches_oracle():
    lx, ly = 8, 12
    rho, ux, uy, T = synth.random_fields(lx, ly, 31, umax=0.08)
    f = M.init_state(rho, ux, uy, T)
    f[:, 3:-3] *= 1.0 + 0.05 * synth.noise(lx, ly, 32)
    p = M.Params(lx, ly, tau=0.75, g=2e-3, t_top=0.85, t_bottom=1.2)
    a = f.copy()
    b = f.copy()
    for _ in range(3):
        a = M.step(a, p)
        b = brute_step(b, lx, ly, p.tau, p.g, p.t_top, p.t_bottom)
    scale = np.abs(M.physical(b)).max(axis=(1, 2), keepdims=True)
    err = np.abs(M.physical(a) - M.physical(b)) / scale
    assert err.max() < 1e-13, err.max()
