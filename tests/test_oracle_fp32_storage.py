"""The float32 shifted storage on its own (CPU): the error floor of any
float32-store arithmetic.

``oracle.storage.step_fp32_storage`` is the float64 oracle step between a
decode and a round-to-nearest encode, so its distance from the float64 oracle
comes from the storage alone.  What the float32 format fixes:

* encode then decode moves a population by at most half a float32 ulp of its
  deviation (plus the float64 rounding of the decode);
* round-to-nearest is unbiased, so over many steps the storage error of the
  density and temperature fields stays flat instead of growing with the step
  count; a biased (truncating) encode leaks mass every step and grows
  linearly, which the same check catches;
* the velocity error stays at the per-step quantum of the momentum sums, a
  few times 1e-8 of the sound speed, however small the velocity itself is.

Lattice: a 32 x 64 Rayleigh-Taylor lattice at the stable contrast
T = 0.75 / 1.25, tau = 0.6, g = 1e-5 (the float32-store error study of the
benchmark at a size the oracle runs in seconds).
"""
import numpy as np
import pytest

import synth
from oracle import lattice, model as M, storage as S

K = lattice.constants()


def _rt(lx=32, ly=64):
    rho, ux, uy, T, tt, tb = synth.rt_fields(lx, ly, 4, 0, delta=0.5)
    p = M.Params(lx, ly, tau=0.6, g=1e-5, t_top=tt, t_bottom=tb)
    return p, M.init_state(rho, ux, uy, T), float(rho.mean())


def test_encode_decode_moves_a_population_by_at_most_half_an_ulp():
    p, f, r0 = _rt()
    f = M.run(f, p, 3)
    d = S.encode(f, r0)
    back = M.physical(S.decode(d, r0))
    dev = M.physical(f) - (K["w"] * r0)[:, None, None]
    half_ulp = 0.5 * np.spacing(np.abs(dev).astype(np.float32)).astype(np.float64)
    assert (np.abs(back - M.physical(f)) <= half_ulp + 4e-16).all()
    assert np.isnan(d[:, :3]).all() and np.isnan(d[:, -3:]).all()


def _errors(fa, fb):
    a, b = M.moments(M.physical(fa)), M.moments(M.physical(fb))
    rel = [np.abs(x - y).max() / np.abs(x).max() for x, y in zip(a, b)]
    absu = max(np.abs(a[1] - b[1]).max(), np.abs(a[2] - b[2]).max())
    return rel, absu


def _storage_run(encode, n_checks=(100, 400)):
    p, f, r0 = _rt()
    d = encode(f, r0)
    f = S.decode(d, r0)
    out = {}
    for n in range(1, max(n_checks) + 1):
        f = M.step(f, p)
        d = encode(M.step(S.decode(d, r0), p), r0)
        if n in n_checks:
            out[n] = _errors(f, S.decode(d, r0))
    return out


def _truncating_encode(f, r0):
    """A biased encode (rounding toward zero): the mistake the flatness check must catch."""
    d = S.encode(f, r0)
    exact = M.physical(f) - (K["w"] * r0)[:, None, None]
    dp = d[:, 3:-3]
    away = np.abs(dp.astype(np.float64)) > np.abs(exact)
    dp[away] = np.nextafter(dp[away], np.float32(0))
    return d


@pytest.mark.slow
def test_storage_rounding_error_is_flat_and_at_the_float32_quantum():
    errs = _storage_run(S.encode)
    for n, (rel, absu) in errs.items():
        rho, _, _, T = rel
        assert rho <= 1e-7 and T <= 1e-7, (n, rel)
        assert absu <= 6e-8, (n, absu)
    # 4x the steps, no growth beyond the noise of the maximum
    assert errs[400][0][0] <= 2.0 * errs[100][0][0] and errs[400][0][3] <= 2.0 * errs[100][0][3], errs


@pytest.mark.slow
def test_a_biased_encode_fails_the_flatness_check():
    errs = _storage_run(_truncating_encode)
    grew = errs[400][0][0] > 2.0 * errs[100][0][0] or errs[400][0][0] > 1e-7
    assert grew, errs
