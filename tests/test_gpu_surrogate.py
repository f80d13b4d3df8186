"""GPU parity of the K* surrogate (tensor-core convolutions, backward, Adam, gate)
against the FP64 oracle in oracle/surrogate.py.

Tolerances. Activations and weights are BF16 (8 significant bits, relative
rounding 2^-9) with FP32 accumulation; six layers of rounding give ~1 % relative
differences in the outputs, so forward outputs are held to 3e-2 relative L2 and
gradients to 5e-2 relative L2 per tensor (with cosine similarity > 0.995). The
patch extraction is FP32 against FP64 (1e-5).
"""

import numpy as np
import pytest

import synth
from oracle import surrogate as S

pytestmark = pytest.mark.gpu


def _lbm():
    import paper_1312_0195_gb300 as lbm
    return lbm


def _t(a, dtype=np.float32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _flat(p):
    parts = []
    for l in range(6):
        parts += [p[f"w{l}"].ravel(), p[f"b{l}"].ravel()]
    parts += [p["wh"].ravel(), p["bh"].ravel()]
    return np.concatenate(parts).astype(np.float32)


def _unflat(v):
    p, o = {}, 0
    for l in range(6):
        ci, co = S.CHANNELS[l], S.CHANNELS[l + 1]
        p[f"w{l}"] = v[o:o + co * ci * 9].reshape(co, ci, 3, 3).astype(np.float64)
        o += co * ci * 9
        p[f"b{l}"] = v[o:o + co].astype(np.float64)
        o += co
    p["wh"] = v[o:o + 128].reshape(2, 64).astype(np.float64)
    o += 128
    p["bh"] = v[o:o + 2].astype(np.float64)
    return p


def _bf16(a):
    """Round to BF16 (round to nearest even) and back, as the device does for inputs and weights."""
    import torch
    return torch.from_numpy(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 2, 32, 32), dtype=np.float32)
    for i in range(n):
        z = synth.gaussian_random_field(32, 32, rng.uniform(2, 8), seed=seed * 100 + i)
        x[i, 0] = rng.normal(-4.0, 0.5) + rng.uniform(0.5, 2.0) * z
        x[i, 1] = np.log2([8, 16, 32, 64][i % 4]) / 6.0
    return x


def test_param_count_matches_oracle_layout():
    lbm = _lbm()
    assert lbm.lbm_surrogate_param_count() == _flat(S.init_params(0)).size == 139266


def test_single_image_forward_matches_oracle():
    """Smallest case first: one image through the network, outputs against the FP64 oracle."""
    lbm = _lbm()
    p = S.init_params(3)
    with lbm.Surrogate(1, 0) as sur:
        sur.set_params(0, _flat(p))
        x = _inputs(1, 1)
        g, loss, y = sur.grad(0, _t(x), _t(np.zeros((1, 2))))
    pq = _unflat(_bf16(_flat(p)))
    yo, _ = S.forward(pq, _bf16(x).astype(np.float64))
    err = np.linalg.norm(y - yo) / max(np.linalg.norm(yo), 1e-12)
    assert err < 3e-2, (y, yo)


def test_forward_and_gradients_match_oracle():
    lbm = _lbm()
    p = S.init_params(7)
    n = 12
    x = _inputs(n, 2)
    t = np.random.default_rng(3).standard_normal((n, 2)).astype(np.float32)
    with lbm.Surrogate(1, 0) as sur:
        sur.set_params(0, _flat(p))
        g, loss, y = sur.grad(0, _t(x), _t(t))
    pq = _unflat(_bf16(_flat(p)))
    yo, cache = S.forward(pq, _bf16(x).astype(np.float64))
    lo, dy = S.mse(yo, t.astype(np.float64))
    go = S.backward(pq, cache, dy)
    assert np.linalg.norm(y - yo) / np.linalg.norm(yo) < 3e-2
    assert abs(loss - lo) <= 3e-2 * lo
    gg = _unflat(g)
    for name in go:
        a, b = gg[name].ravel(), go[name].ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-20)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        assert rel < 5e-2 and cos > 0.995, (name, rel, cos)


def test_adam_step_matches_oracle():
    """One training step (batch = all samples) is one Adam update of the FP32 master weights
    with the step's gradient; checked against the oracle's Adam on the GPU's own gradient."""
    lbm = _lbm()
    p = S.init_params(11)
    n = 8
    x = _inputs(n, 4)
    ylab = np.random.default_rng(5).normal(-3.0, 0.7, size=(n, 2)).astype(np.float32)
    stats = np.stack([S.patch_stats(x[i, 0].astype(np.float64)) for i in range(n)]).astype(np.float32)
    with lbm.Surrogate(1, 0) as sur:
        sur.set_params(0, _flat(p))
        norm0 = sur.get_normalization()
        norm0[12] = 0                          # targets relative to the patch's mean log K (rebuilt below)
        sur.set_normalization(norm0)
        sur.train(_t(x), _t(ylab), _t(stats), epochs=1, batch=n, lr=1e-3, seed=0)
        p1 = sur.get_params(0)
        norm = sur.get_normalization()
        # the same step's gradient, with the normalisation train() chose
        sur.set_params(0, _flat(p))
        pm = x[:, 0].mean(axis=(1, 2))        # targets are learned relative to the patch's mean log K
        tstd = np.stack([(ylab[:, 0] - pm - norm[2]) / norm[3], (ylab[:, 1] - pm - norm[4]) / norm[5]], axis=1)
        g, _, _ = sur.grad(0, _t(x), _t(tstd))
    ref, _, _ = S.adam_step(_flat(p).astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    # training sums the batch in its own shuffled order, so gradients that are pure
    # rounding noise (|g| tiny) may flip sign; everything well above that must agree
    sig = np.abs(g) > 1e-4 * np.abs(g).max()
    assert sig.mean() > 0.5
    np.testing.assert_allclose(p1[sig], ref[sig], rtol=0, atol=2e-6)
    assert (np.abs(p1 - ref) <= 2.1e-3).all()
    # input normalisation = mean / std of the log-K plane over the data
    assert abs(norm[0] - x[:, 0].mean()) < 1e-4 and abs(norm[1] - x[:, 0].std()) < 1e-4


def test_patches_match_oracle():
    import torch
    lbm = _lbm()
    kap = synth.lognormal_kappa(128, 128, 6.0, 1.5, seed=9).astype(np.float32)
    leaves = np.array([[0, 0, 8], [8, 0, 16], [32, 32, 32], [64, 64, 64], [100, 4, 4]], dtype=np.int32)
    x, st = lbm.lbm_patches(_t(kap), torch.from_numpy(leaves).cuda())
    x, st = x.cpu().numpy(), st.cpu().numpy()
    for i, (x0, y0, s) in enumerate(leaves):
        ref = S.resample_patch(np.log(kap[y0:y0 + s, x0:x0 + s].astype(np.float64)))
        np.testing.assert_allclose(x[i, 0], ref, rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(x[i, 1], np.log2(s) / 6.0, rtol=1e-6)
        np.testing.assert_allclose(st[i], S.patch_stats(ref), rtol=1e-4, atol=1e-5)


def test_training_fits_a_smooth_target():
    """Training mechanics: on a learnable target (mean and spread of log K) the loss falls by 10x."""
    lbm = _lbm()
    n = 512
    x = _inputs(n, 6)
    y = np.stack([x[:, 0].mean(axis=(1, 2)), x[:, 0].std(axis=(1, 2)) + 0.3 * x[:, 1, 0, 0]], axis=1)
    stats = np.zeros((n, 3), dtype=np.float32)
    with lbm.Surrogate(2, 1) as sur:
        norm = sur.get_normalization()
        assert norm[12] == 2                          # a new ensemble learns the bound-normalised target
        norm[12] = 0                                  # mechanics only: the plain mean-log-K base
        sur.set_normalization(norm)
        loss = sur.train(_t(x), _t(y), _t(stats), epochs=30, batch=64, lr=2e-3, seed=1)
        pred = sur.predict(_t(x)).cpu().numpy()
    print("training loss per epoch (model 0):", loss[0][::5])
    assert loss[0][-1] < 0.1 * loss[0][0] and loss[1][-1] < 0.1 * loss[1][0]
    err = np.abs(pred.mean(axis=0) - y)
    assert np.median(err[:, 0]) < 0.1


def test_gate_routes_blocks():
    """spread_max tiny -> every block falls back to local LBM; the result then equals the LBM-only
    upscaling. A generous gate accepts in-range blocks and returns exp(ensemble mean)."""
    import torch
    lbm = _lbm()
    kap = synth.lognormal_kappa(64, 64, 6.0, 1.0, seed=12).astype(np.float32)
    p = lbm.Params(nx=64, ny=64, tau=1.0, eps=1.0)
    kt = _t(kap)
    with lbm.Surrogate(3, 5) as sur:
        norm = np.array([-4.6, 1.0, -4.6, 1.0, -4.6, 1.0, -1e9, 1e9, -1e9, 1e9, -1e9, 1e9, 0], dtype=np.float32)
        sur.set_normalization(norm)
        k_lbm = torch.empty((4, 4, 4), dtype=torch.float64, device="cuda")
        k_fb = torch.empty_like(k_lbm)
        k_sur = torch.empty_like(k_lbm)
        lbm.lbm_upscale(p, kt, 16, k_lbm, 1e-6, 0.0, 320)
        st, nfb = lbm.lbm_upscale(p, kt, 16, k_fb, 1e-6, 0.0, 320, surrogate=sur, spread_max=1e-30)
        assert nfb == 16
        assert torch.equal(k_fb, k_lbm)
        st, nfb = lbm.lbm_upscale(p, kt, 16, k_sur, 1e-6, 0.0, 320, surrogate=sur, spread_max=1e30)
        assert nfb == 0
        leaves = torch.from_numpy(synth.uniform_leaves(64, 64, 16)).cuda()
        x, _ = lbm.lbm_patches(kt, leaves)
        pred = sur.predict(x).cpu().numpy()
    ks = k_sur.cpu().numpy().reshape(16, 4)
    np.testing.assert_allclose(ks[:, 0], np.exp(pred[:, :, 0].mean(axis=0)), rtol=1e-5)
    np.testing.assert_allclose(ks[:, 3], np.exp(pred[:, :, 1].mean(axis=0)), rtol=1e-5)
    assert (ks[:, 1] == 0).all() and (ks[:, 2] == 0).all()


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_target_base_modes(mode):
    """With every weight zero and target mean 0 the network contributes nothing, so the prediction is
    the per-patch base c of the target mode. Mode 0: mean log K. Modes 1 and 2: the midpoint of the
    layered-medium bounds, which for a patch of layers across x collapse to the harmonic mean of the
    layers for K*_xx and their arithmetic mean for K*_yy (Tables 1 and 2 in the Darcy limit)."""
    import torch
    lbm = _lbm()
    rng = np.random.default_rng(81)
    layers = np.exp(rng.uniform(-6.0, 0.0, 32))                    # K varies along x only
    logk = [np.tile(np.log(layers), (32, 1)), rng.normal(-3.0, 1.2, (32, 32))]
    x = np.zeros((2, 2, 32, 32), dtype=np.float32)
    for i, lk in enumerate(logk):
        x[i, 0] = lk
        x[i, 1] = 5.0 / 6.0
    with lbm.Surrogate(1, 0) as sur:
        sur.set_params(0, np.zeros(lbm.lbm_surrogate_param_count(), dtype=np.float32))
        norm = np.array([0, 1, 0, 1, 0, 1, -1e30, 1e30, -1e30, 1e30, -1e30, 1e30, mode], dtype=np.float32)
        sur.set_normalization(norm)
        y = sur.predict(torch.from_numpy(x).cuda()).cpu().numpy()[0]
    for i, lk in enumerate(logk):
        k = np.exp(lk.astype(np.float32).astype(np.float64))
        if mode == 0:
            cx = cy = lk.astype(np.float32).astype(np.float64).mean()
        else:
            lox = np.log((1.0 / (1.0 / k).mean(axis=1)).mean())        # rows (series along x) in parallel
            hix = np.log(1.0 / (1.0 / k.mean(axis=0)).mean())          # columns (parallel) in series
            loy = np.log((1.0 / (1.0 / k).mean(axis=0)).mean())
            hiy = np.log(1.0 / (1.0 / k.mean(axis=1)).mean())
            cx, cy = 0.5 * (lox + hix), 0.5 * (loy + hiy)
        np.testing.assert_allclose(y[i], [cx, cy], rtol=0, atol=2e-5)
    if mode:
        np.testing.assert_allclose(y[0, 0], np.log(1.0 / (1.0 / layers.astype(np.float32)).mean()), atol=2e-5)
        np.testing.assert_allclose(y[0, 1], np.log(layers.astype(np.float32).mean()), atol=2e-5)
    with lbm.Surrogate(1, 0) as sur, pytest.raises(lbm.LbmError):
        sur.set_normalization(np.array([0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 3], dtype=np.float32))
