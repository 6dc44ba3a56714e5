"""The seeded inputs follow the stated recipe (CPU only): the Rayleigh-Taylor
initial condition at rest in pressure balance with a cold dense upper layer,
seeded and reproducible, and batches drawn from the stated ranges."""
import numpy as np

import synth


def test_rayleigh_taylor_fields_follow_the_recipe():
    lx, ly = 256, 128
    rho, ux, uy, T, t_top, t_bottom = synth.rt_fields(lx, ly, 32, seed=0)
    assert rho.shape == ux.shape == uy.shape == T.shape == (ly, lx)
    assert not ux.any() and not uy.any()                       # at rest
    np.testing.assert_allclose(rho * T, 1.0, rtol=1e-15)      # isobaric, p0 = 1
    assert (t_top, t_bottom) == (0.5, 1.5)                     # walls take the far-field temperatures
    assert T.min() >= 0.5 and T.max() <= 1.5
    np.testing.assert_allclose(T[-1], 0.5, atol=1e-9)         # cold on top (interface amplitude <= 2 * modes)
    np.testing.assert_allclose(T[0], 1.5, atol=1e-9)
    # the interface (T = 1 crossing) sits at ly/2 + sum of at most 32 cosines of amplitude <= 2
    crossing = np.argmin(np.abs(T - 1.0), axis=0)
    assert np.abs(crossing - ly / 2).max() <= 2 * 32 + 1
    assert crossing.std() > 0.5                                # perturbed, not flat


def test_rayleigh_taylor_fields_are_seeded():
    a = synth.rt_fields(64, 128, 4, seed=3)
    b = synth.rt_fields(64, 128, 4, seed=3)
    c = synth.rt_fields(64, 128, 4, seed=4)
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(a[3], c[3])


def test_smaller_contrast_keeps_the_far_field_temperatures():
    _, _, _, T, t_top, t_bottom = synth.rt_fields(64, 64, 4, seed=1, delta=0.5)
    assert (t_top, t_bottom) == (0.75, 1.25)
    assert T.min() >= 0.75 and T.max() <= 1.25


def test_batch_draws_from_the_stated_ranges():
    specs = synth.batch_lattices(64, seed=0)
    assert len(specs) == 64
    assert {s.lx for s in specs} <= {128, 256, 512, 1024}
    assert {s.ly for s in specs} <= {256, 512, 1024, 2048}
    assert len({(s.lx, s.ly) for s in specs}) > 8                # uneven sizes
    for s in specs:
        assert 0.55 <= s.tau <= 1.0 and 1e-5 <= s.g <= 1e-4 and 0.2 <= s.delta <= 1.0
    assert [s.seed for s in synth.batch_lattices(64, seed=0)] == [s.seed for s in specs]
