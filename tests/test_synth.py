"""Seeded input generators: determinism, coverage and the statistics they promise."""

import numpy as np

import synth


def test_grf_standardised_and_seeded():
    z = synth.gaussian_random_field(128, 64, 8.0, seed=1)
    assert z.shape == (64, 128)
    assert abs(z.mean()) < 1e-12 and abs(z.std() - 1.0) < 1e-12
    np.testing.assert_array_equal(z, synth.gaussian_random_field(128, 64, 8.0, seed=1))
    assert not np.array_equal(z, synth.gaussian_random_field(128, 64, 8.0, seed=2))


def test_grf_correlation_length():
    """Empirical correlation at lag ell is near exp(-1/2) for C(r) = exp(-r^2 / (2 ell^2))."""
    ell = 16.0
    z = synth.gaussian_random_field(1024, 1024, ell, seed=7)
    lag = int(ell)
    c = np.mean(z * np.roll(z, lag, axis=1))
    assert abs(c - np.exp(-0.5)) < 0.05


def test_quadtree_covers_field_once():
    leaves = synth.quadtree_leaves(512, 256, seed=3)
    cover = np.zeros((256, 512), dtype=np.int32)
    for x0, y0, s in leaves:
        assert s in (8, 16, 32, 64)
        assert x0 % s == 0 and y0 % s == 0
        cover[y0:y0 + s, x0:x0 + s] += 1
    assert cover.min() == 1 and cover.max() == 1
    np.testing.assert_array_equal(leaves, synth.quadtree_leaves(512, 256, seed=3))


def test_quadtree_expected_leaf_count():
    """p = 0.6 gives 17.49 expected leaves per 64-cell root."""
    leaves = synth.quadtree_leaves(2048, 2048, seed=3)
    per_root = len(leaves) / (32 * 32)
    assert abs(per_root - 17.49) < 0.6


def test_paper_fields():
    k = synth.block_kappa_eq22()
    assert (k == 1e-6).sum() == 40 * 40 and k[30, 30] == 1e-6 and k[29, 30] == 1e-5
    lay = synth.layered_kappa(100, 3, 1.0, 5.0)
    assert lay[0, 0] == 1.0 and lay[0, 10] == 5.0 and lay[2, 95] == 5.0
    cb = synth.checkerboard_kappa(100, 1.0, 2.0)
    assert cb[0, 0] == 1.0 and cb[0, 10] == 2.0 and cb[10, 10] == 1.0
    f = synth.fiveblock_kappa_eq23(400, 1.0)
    c = synth.fiveblock_coarse_kappa_eq24(40, 1.0, 8.485)
    # blocks of Eq. 23 land exactly on the coarse blocks of Eq. 24
    fine_const = (f == 1.0).reshape(40, 10, 40, 10).all(axis=(1, 3))
    np.testing.assert_array_equal(fine_const, c == 1.0)
    g = synth.sinusoidal_g_field(40, 2.0)
    assert g.shape == (2, 40, 40) and abs(g[0, 0, 20] - 2.0 * np.sin(np.pi * 20.5 / 40)) < 1e-14


def test_channel_field_contrast():
    k = synth.channel_kappa(1024, 1024, seed=5)
    vals = set(np.unique(k).tolist())
    assert vals == {np.float32(1e-6).item(), np.float32(1e-2).item()}
    frac = (k == np.float32(1e-2)).mean()
    assert 0.02 < frac < 0.2


def test_crop_periodic_wraps():
    a = np.arange(20).reshape(4, 5)
    c = synth.crop_periodic(a, 3, 2, 4, 3)
    assert c.shape == (3, 4)
    assert c[0, 0] == a[2, 3] and c[0, 2] == a[2, 0] and c[2, 0] == a[0, 3]
