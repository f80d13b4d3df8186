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
    x = RNG.standard_normal((2, 2, 32, 32))
    y, (acts, pooled) = S.forward(p, x)
    assert y.shape == (2, 2) and pooled.shape == (2, 64) and len(acts) == 7
    np.testing.assert_allclose(y, pooled @ p["wh"].T + p["bh"], rtol=1e-14)
