"""Pins of the FP64 surrogate oracle (CPU only)."""

import numpy as np
import pytest

from oracle import surrogate as S

RNG = np.random.default_rng(2024)


def test_conv3x3_matches_scipy_correlate():
    scipy_signal = pytest.importorskip("scipy.signal")
    x = RNG.standard_normal((2, 3, 7, 9))
    w = RNG.standard_normal((4, 3, 3, 3))
    b = RNG.standard_normal(4)
    y = S.conv3x3(x, w, b)
    ref = np.zeros_like(y)
    for n in range(2):
        for o in range(4):
            acc = np.full((7, 9), b[o])
            for c in range(3):
                acc += scipy_signal.correlate2d(x[n, c], w[o, c], mode="same", boundary="fill", fillvalue=0.0)
            ref[n, o] = acc
    np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-13)


def test_backward_matches_central_differences():
    """dL/dtheta of the oracle against (L(theta + h) - L(theta - h)) / 2h, h = 1e-6, on a small net."""
    ch = (2, 3, 4)
    p = S.init_params(5, ch)
    x = RNG.standard_normal((3, 2, 6, 6))
    t = RNG.standard_normal((3, 2))

    def loss(pp):
        y, _ = S.forward(pp, x, nlayers=2)
        return S.mse(y, t)[0]

    y, cache = S.forward(p, x, nlayers=2)
    _, dy = S.mse(y, t)
    g = S.backward(p, cache, dy, nlayers=2)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        idx = RNG.choice(flat.size, min(6, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = loss(p)
            flat[i] = old - h
            lm = loss(p)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, i, fd, an)


def test_adam_first_step_is_signed_lr():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is -lr g / (|g| + eps)."""
    th = RNG.standard_normal(10)
    g = RNG.standard_normal(10)
    new, m, v = S.adam_step(th, g, np.zeros(10), np.zeros(10), 1, 1e-3)
    np.testing.assert_allclose(new, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(m, 0.1 * g, rtol=1e-12)
    np.testing.assert_allclose(v, 0.001 * g * g, rtol=1e-12)


def test_resample_and_stats():
    a = RNG.standard_normal((8, 8))
    p = S.resample_patch(a)
    assert p.shape == (32, 32) and np.array_equal(p[::4, ::4], a) and np.array_equal(p[3::4, 3::4], a)
    b = RNG.standard_normal((64, 64))
    q = S.resample_patch(b)
    np.testing.assert_allclose(q[5, 7], b[10:12, 14:16].mean(), rtol=1e-14)
    c = np.full((32, 32), 1.5)
    np.testing.assert_allclose(S.patch_stats(c), [1.5, 0.0, 0.0], atol=1e-15)
    ramp = np.add.outer(np.zeros(32), 0.25 * np.arange(32))
    st = S.patch_stats(ramp)
    assert abs(st[2] - 0.5 * 0.25 ** 2) < 1e-14


def test_forward_shapes_and_pool_linearity():
    p = S.init_params(1)
    x = RNG.standard_normal((2, 9, 32, 32))
    y, (acts, pooled) = S.forward(p, x)
    assert y.shape == (2, 2) and pooled.shape == (2, 64) and len(acts) == 7
    np.testing.assert_allclose(y, pooled @ p["wh"].T + p["bh"], rtol=1e-14)


# ------------------------------------------------------------ leaf planes, target base, gate

def test_phase_planes_carry_every_cell():
    """A 64-cell leaf is split by row and column parity with nothing lost; a leaf of 32 cells or
    fewer appears as four equal copies of its replicated patch; 128 cells are 2 x 2 block means."""
    b = RNG.standard_normal((64, 64))
    ph = S.phase_planes(b)
    assert ph.shape == (4, 32, 32)
    rebuilt = np.empty((64, 64))
    for a in (0, 1):
        for c in (0, 1):
            rebuilt[a::2, c::2] = ph[2 * a + c]
    assert np.array_equal(rebuilt, b)
    a8 = RNG.standard_normal((8, 8))
    ph8 = S.phase_planes(a8)
    for k in range(4):
        assert np.array_equal(ph8[k], np.kron(a8, np.ones((4, 4))))
    big = RNG.standard_normal((128, 128))
    np.testing.assert_allclose(S.full_plane(big)[3, 5], big[6:8, 10:12].mean(), rtol=1e-14)
    for bad in (48, 96, 0):
        with pytest.raises(ValueError):
            S.phase_planes(np.zeros((bad, bad)))
    x = S.make_input(np.log(np.full((16, 16), 0.01)), np.log(0.01), 2.0)
    assert np.array_equal(x[:4], np.zeros((4, 32, 32))) and np.all(x[4] == 4.0 / 6.0)
    assert np.abs(x[5:]).max() < 1e-15


def test_layered_bounds_reproduce_tables_1_and_2():
    """Layers across x (K varies along x only): flow along x crosses them in series, so both
    bounds are the harmonic mean (Table 1's analytic column); flow along y runs along them in
    parallel, so both are the arithmetic mean (Table 2's). Checked against scipy's means."""
    stats = pytest.importorskip("scipy.stats")
    layers = np.exp(RNG.uniform(-7.0, 0.0, 64))
    logk = np.tile(np.log(layers), (64, 1))
    lox, hix, loy, hiy = S.layered_bounds(np.exp(logk))
    hm, am = stats.hmean(layers), np.mean(layers)
    np.testing.assert_allclose([lox, hix], [hm, hm], rtol=1e-13)
    np.testing.assert_allclose([loy, hiy], [am, am], rtol=1e-13)
    cx, wx, cy, wy = S.target_base(logk, 2)
    np.testing.assert_allclose([cx, cy], [np.log(hm), np.log(am)], rtol=0, atol=1e-13)
    assert wx == 0.05 and wy == 0.05          # collapsed bounds: the width floor
    # the same layers seen by the 8 x 8 and 32 x 32 paths of full_plane (repetition keeps means)
    k8 = np.tile(np.log(layers[::8]), (8, 1))
    c8 = S.target_base(k8, 1)
    np.testing.assert_allclose(c8[0], np.log(stats.hmean(layers[::8])), atol=1e-13)
    np.testing.assert_allclose(c8[2], np.log(np.mean(layers[::8])), atol=1e-13)


def test_checkerboard_base_is_the_geometric_mean_of_table_3():
    """On a checkerboard of two permeabilities both the series-of-rows and parallel-of-columns
    arrangements mix k1 and k2 half and half, so the bounds are their harmonic and arithmetic
    means, whose log midpoint is log sqrt(k1 k2): Table 3's analytic value."""
    for k1, k2 in ((1.0, 2.0), (1.0, 100.0), (3e-3, 7e-6)):
        idx = np.add.outer(np.arange(64) // 8, np.arange(64) // 8) % 2
        logk = np.where(idx == 0, np.log(k1), np.log(k2))
        lox, hix, loy, hiy = S.layered_bounds(np.exp(logk))
        np.testing.assert_allclose([lox, hix], [2 * k1 * k2 / (k1 + k2), 0.5 * (k1 + k2)], rtol=1e-12)
        cx, wx, cy, wy = S.target_base(logk, 2)
        np.testing.assert_allclose([cx, cy], [0.5 * np.log(k1 * k2)] * 2, rtol=0, atol=1e-12)
        np.testing.assert_allclose(wx, max(0.5 * np.log((k1 + k2) ** 2 / (4 * k1 * k2)), 0.05), rtol=1e-12)


def test_target_base_symmetries_and_modes():
    """Transposing a patch exchanges the xx and yy bases; a uniform patch gives log K with the
    width floor; lo <= hi on random patches; mode 0 is the mean log K and mode 1 has w = 1."""
    logk = RNG.normal(-4.0, 1.5, (64, 64))
    a = S.target_base(logk, 2)
    b = S.target_base(logk.T.copy(), 2)
    np.testing.assert_allclose([a[2], a[3], a[0], a[1]], b, rtol=1e-13)
    lox, hix, loy, hiy = S.layered_bounds(np.exp(logk))
    assert lox < hix and loy < hiy
    assert a[1] > 0.05 and a[3] > 0.05
    u = S.target_base(np.full((32, 32), np.log(0.02)), 2)
    np.testing.assert_allclose(u, [np.log(0.02), 0.05, np.log(0.02), 0.05], rtol=1e-14)
    m0 = S.target_base(logk, 0)
    np.testing.assert_allclose(m0, [logk.mean(), 1.0, logk.mean(), 1.0], rtol=1e-14)
    m1 = S.target_base(logk, 1)
    np.testing.assert_allclose([m1[0], m1[2]], [a[0], a[2]], rtol=1e-14)
    assert m1[1] == 1.0 and m1[3] == 1.0


def test_gate_hand_made_spreads():
    """Four members at c +- d (two each) have sample standard deviation d sqrt(4/3): at the 3 %
    gate (threshold ln 1.03 = 0.0295588) d = 0.0255 passes and d = 0.0257 fails. Statistics on
    the bounds pass, a hair outside fails; a NaN member fails; one member has spread 0. The
    accepted K* is the geometric mean of the members' K*."""
    stats = pytest.importorskip("scipy.stats")
    thr = np.log(1.03)
    assert 0.0255 * np.sqrt(4 / 3) < thr < 0.0257 * np.sqrt(4 / 3)
    c = np.array([-4.2, -3.1])
    pat = np.array([1.0, -1.0, 1.0, -1.0])
    ys = []
    for d in (0.0255, 0.0257, 0.0):
        ys.append(c[None, :] + d * pat[:, None] * np.array([[1.0, 0.3]]))
    ys.append(np.array([[-4.0, -3.0], [np.nan, -3.0], [-4.0, -3.0], [-4.0, -3.0]]))
    y = np.stack(ys, axis=1)                     # [4][4][2]
    lo, hi = np.array([-5.0, 0.1, 0.0]), np.array([-1.0, 2.0, 1.0])
    st = np.array([[-3.0, 1.0, 0.5]] * 4)
    acc, keff = S.gate(y, st, np.full(4, 16), lo, hi, 0.03)
    assert acc.tolist() == [True, False, True, False]
    np.testing.assert_allclose(keff[0], [stats.gmean(np.exp(y[:, 0, 0])), 0, 0, stats.gmean(np.exp(y[:, 0, 1]))],
                               rtol=1e-14)
    assert np.isnan(keff[1]).all()
    # statistics: bounds are inclusive
    st2 = np.array([[-5.0, 2.0, 1.0], [-5.0 - 1e-12, 1.0, 0.5], [-3.0, 0.1 - 1e-12, 0.5], [-3.0, 1.0, 1.0 + 1e-12]])
    y2 = np.repeat(ys[2][:, None, :], 4, axis=1)
    acc2, _ = S.gate(y2, st2, np.full(4, 8), lo, hi, 0.03)
    assert acc2.tolist() == [True, False, False, False]
    # per-size thresholds: the same leaf passes at 8 cells and fails at 64
    acc3, _ = S.gate(np.repeat(ys[0][:, None, :], 2, axis=1), st[:2], np.array([8, 64]), lo, hi, {8: 0.03, 64: 0.02})
    assert acc3.tolist() == [True, False]
    # a single member has no spread
    acc4, keff4 = S.gate(y[:1, :1], st[:1], np.array([32]), lo, hi, 1e-9)
    assert acc4.tolist() == [True] and keff4[0, 0] == np.exp(y[0, 0, 0])


def test_context_planes_are_row_and_column_means():
    """A patch of layers across x: every row has the same series (harmonic) and parallel
    (arithmetic) mean along x; each column is uniform, so its means along y are its own value.
    Checked against scipy's means; transposing the patch exchanges the row and column planes."""
    stats = pytest.importorskip("scipy.stats")
    layers = np.exp(RNG.uniform(-6.0, 0.0, 32))
    p = np.tile(np.log(layers), (32, 1))
    c = S.context_planes(p)
    np.testing.assert_allclose(c[0], np.log(stats.hmean(layers)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(c[1], np.log(np.mean(layers)), rtol=0, atol=1e-13)
    np.testing.assert_allclose(c[2], p, rtol=0, atol=1e-13)
    np.testing.assert_allclose(c[3], p, rtol=0, atol=1e-13)
    q = RNG.normal(-3.0, 1.0, (32, 32))
    a, b = S.context_planes(q), S.context_planes(q.T.copy())
    np.testing.assert_allclose(b[0], a[2].T, rtol=1e-13)
    np.testing.assert_allclose(b[3], a[1].T, rtol=1e-13)
    x = S.make_input(q, -3.0, 2.0)
    assert x.shape == (9, 32, 32)
    np.testing.assert_allclose(x[5:], (a - (-3.0)) / 2.0, rtol=1e-14)


def test_darcy_keff_closed_forms():
    """Finite-volume Darcy K* of a periodic patch: a uniform patch gives its permeability; layers
    across x give the harmonic mean along x and the arithmetic mean along y exactly (Tables 1 and
    2's analytic columns); on a checkerboard of single cells every face has the same harmonic
    permeability 2 k1 k2 / (k1 + k2), which is then K* in both directions; transposing a random
    patch exchanges K*_xx and K*_yy and a periodic shift changes nothing."""
    stats = pytest.importorskip("scipy.stats")
    np.testing.assert_allclose(S.darcy_keff(np.full((8, 8), 0.3)), [0.3, 0.3], rtol=1e-13)
    layers = np.exp(RNG.uniform(-6.0, 0.0, 16))
    kxx, kyy = S.darcy_keff(np.tile(layers, (16, 1)))
    np.testing.assert_allclose([kxx, kyy], [stats.hmean(layers), np.mean(layers)], rtol=1e-11)
    for k1, k2 in ((1.0, 2.0), (3e-3, 7e-6)):
        idx = np.add.outer(np.arange(12), np.arange(12)) % 2
        kc = np.where(idx == 0, k1, k2)
        np.testing.assert_allclose(S.darcy_keff(kc), [2 * k1 * k2 / (k1 + k2)] * 2, rtol=1e-11)
    q = np.exp(RNG.normal(-3.0, 1.5, (16, 16)))
    a, b = S.darcy_keff(q), S.darcy_keff(q.T.copy())
    np.testing.assert_allclose([a[1], a[0]], b, rtol=1e-11)
    np.testing.assert_allclose(S.darcy_keff(np.roll(q, (5, 3), axis=(0, 1))), a, rtol=1e-11)
    # lies between the layered bounds of Tables 1 and 2 (harmonic of arithmetic, arithmetic of harmonic)
    lox, hix, loy, hiy = S.layered_bounds(q)
    assert lox <= a[0] <= hix and loy <= a[1] <= hiy
    # mode 3 of the target base is its log (the leaf itself, width 1)
    np.testing.assert_allclose(S.target_base(np.log(q), 3), [np.log(a[0]), 1.0, np.log(a[1]), 1.0], rtol=1e-13)
