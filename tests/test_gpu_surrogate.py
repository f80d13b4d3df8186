"""GPU parity of the K* surrogate (tensor-core convolutions, backward, Adam, gate)
against the FP64 oracle in oracle/surrogate.py.

Tolerances. Activations and weights are BF16 (8 significant bits, relative
rounding 2^-9) with FP32 accumulation; six layers of rounding give ~1 % relative
differences in the outputs, so forward outputs are held to 3e-2 relative L2 and
gradients to 5e-2 relative L2 per tensor (with cosine similarity > 0.995). The
patch extraction is FP32 against FP64 (1e-5). The gate takes its decisions in FP64 on
both sides from the same FP32 member outputs, so decisions and accepted K* must agree
exactly (K* to the last bits of exp).

Sizes. A tensor-core convolution launch holds at most 152 x (CTAs per SM) persistent
CTAs, each taking half-image work items in turn; the full-batch cases (512 and 640
images) give every CTA three or more items, so the double-buffered input stages and
TMEM accumulators are each reused and their mbarrier phases flip, and the weight-
gradient kernels fold many items per CTA.
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


def _leaves_logk(n, seed):
    """n seeded log-permeability leaves of 8, 16, 32 and 64 cells (Gaussian random fields)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        s = [8, 16, 32, 64][i % 4]
        z = synth.gaussian_random_field(s, s, rng.uniform(1.5, 8), seed=seed * 1000 + i)
        out.append(rng.normal(-4.0, 0.5) + rng.uniform(0.5, 2.0) * z)
    return out


def _inputs(n, seed, leaves=None):
    """Surrogate inputs [n, 9, 32, 32] of the oracle (log-K planes unnormalised)."""
    leaves = _leaves_logk(n, seed) if leaves is None else leaves
    return np.stack([S.make_input(lk, 0.0, 1.0) for lk in leaves]).astype(np.float32)


def test_param_count_matches_oracle_layout():
    lbm = _lbm()
    assert lbm.lbm_surrogate_param_count() == _flat(S.init_params(0)).size == 141282


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
    stats = np.stack([S.patch_stats(x[i, :4].astype(np.float64).mean(axis=0)) for i in range(n)]).astype(np.float32)
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
        pm = x[:, :4].astype(np.float64).mean(axis=(1, 2, 3))   # targets relative to the leaf's mean log K
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
    assert abs(norm[0] - x[:, :4].mean()) < 1e-4 and abs(norm[1] - x[:, :4].std()) < 1e-4


def test_patches_match_oracle():
    """Nine planes per leaf against the oracle: the four phase planes of the leaf's 64 x 64 log-K
    plane (a 64-cell leaf at full resolution, a 128-cell one as 2 x 2 means, smaller ones
    repeated), the size plane, the four row and column context planes, and the statistics of the
    32 x 32 mean patch."""
    import torch
    lbm = _lbm()
    kap = synth.lognormal_kappa(128, 128, 6.0, 1.5, seed=9).astype(np.float32)
    leaves = np.array([[0, 0, 8], [8, 0, 16], [32, 32, 32], [64, 64, 64], [100, 4, 4], [0, 0, 128], [3, 5, 1]],
                      dtype=np.int32)
    x, st = lbm.lbm_patches(_t(kap), torch.from_numpy(leaves).cuda())
    x, st = x.cpu().numpy(), st.cpu().numpy()
    for i, (x0, y0, s) in enumerate(leaves):
        lk = np.log(kap[y0:y0 + s, x0:x0 + s].astype(np.float64))
        np.testing.assert_allclose(x[i, :4], S.phase_planes(lk), rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(x[i, 4], np.log2(s) / 6.0, rtol=1e-6)
        # context of the FP32 mean patch the device forms
        pm = x[i, :4].astype(np.float64).mean(axis=0)
        np.testing.assert_allclose(x[i, 5:], S.context_planes(pm), rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(st[i], S.patch_stats(S.resample_patch(lk)), rtol=1e-4, atol=1e-5)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_patches(_t(kap), torch.tensor([[0, 0, 96]], dtype=torch.int32, device="cuda"))


def test_training_fits_a_smooth_target():
    """Training mechanics: on a learnable target (mean and spread of log K) the loss falls by 10x."""
    lbm = _lbm()
    n = 512
    x = _inputs(n, 6)
    y = np.stack([x[:, :4].mean(axis=(1, 2, 3)), x[:, :4].std(axis=(1, 2, 3)) + 0.3 * x[:, 4, 0, 0]], axis=1)
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


def _base_from_predict(sur, x, mode, n_models=1):
    """(c, w) per leaf as the library computes them: with every weight zero the network outputs 0,
    so the prediction is c + w * mean; two calls with target means 0 and 1 give c and w."""
    import torch
    lbm = _lbm()
    for m in range(n_models):
        sur.set_params(m, np.zeros(lbm.lbm_surrogate_param_count(), dtype=np.float32))
    out = []
    for mean in (0.0, 1.0):
        norm = np.array([0, 1, mean, 1, mean, 1, -1e30, 1e30, -1e30, 1e30, -1e30, 1e30, mode], dtype=np.float32)
        sur.set_normalization(norm)
        out.append(sur.predict(torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()[0].astype(np.float64))
    c, cw = out
    return c, cw - c


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_target_base_matches_oracle_full_batch(mode):
    """The per-leaf base (c, w) of every target mode against the oracle's target_base on 640
    leaves of 8 to 64 cells, plus layers across x (the Table 1 and 2 means, exact for the layered
    bounds and for the finite-volume Darcy K* of mode 3) and a checkerboard (Table 3's geometric
    mean for the bounds' midpoint)."""
    lbm = _lbm()
    leaves = _leaves_logk(640, 31)
    layers = np.exp(np.random.default_rng(81).uniform(-6.0, 0.0, 64))
    leaves[0] = np.tile(np.log(layers), (64, 1))
    idx = np.add.outer(np.arange(32) // 4, np.arange(32) // 4) % 2
    leaves[2] = np.where(idx == 0, np.log(1e-3), np.log(2e-2))
    x = _inputs(len(leaves), 0, leaves)
    with lbm.Surrogate(1, 0) as sur:
        c, w = _base_from_predict(sur, x, mode)
    # the oracle sees what the device sees: the leaf's log K rounded to FP32, as in x
    ref = np.array([S.target_base(lk.astype(np.float32).astype(np.float64), mode) for lk in leaves])
    np.testing.assert_allclose(c[:, 0], ref[:, 0], rtol=0, atol=3e-5)
    np.testing.assert_allclose(c[:, 1], ref[:, 2], rtol=0, atol=3e-5)
    np.testing.assert_allclose(w[:, 0], ref[:, 1], rtol=3e-5, atol=3e-6)
    np.testing.assert_allclose(w[:, 1], ref[:, 3], rtol=3e-5, atol=3e-6)
    if mode:
        l32 = layers.astype(np.float32).astype(np.float64)
        np.testing.assert_allclose(c[0], [np.log(1.0 / (1.0 / l32).mean()), np.log(l32.mean())], atol=3e-5)
    if mode in (1, 2):
        np.testing.assert_allclose(c[2], [0.5 * np.log(1e-3 * 2e-2)] * 2, atol=3e-5)
    with lbm.Surrogate(1, 0) as sur, pytest.raises(lbm.LbmError):
        sur.set_normalization(np.array([0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 0, 1, 4], dtype=np.float32))


def test_full_batch_forward_and_gradients_match_oracle():
    """512 images in one forward + backward pass: the network outputs and every gradient tensor
    against the FP64 oracle, with each persistent CTA of the convolutions taking several items."""
    lbm = _lbm()
    p = S.init_params(17)
    n = 512
    x = _inputs(n, 12)
    t = np.random.default_rng(13).standard_normal((n, 2)).astype(np.float32)
    with lbm.Surrogate(1, 0) as sur:
        sur.set_params(0, _flat(p))
        g, loss, y = sur.grad(0, _t(x), _t(t))
    pq = _unflat(_bf16(_flat(p)))
    yo, cache = S.forward(pq, _bf16(x).astype(np.float64))
    lo, dy = S.mse(yo, t.astype(np.float64))
    go = S.backward(pq, cache, dy)
    err = np.linalg.norm(y - yo) / np.linalg.norm(yo)
    print(f"512-image forward rel L2 {err:.2e}")
    assert err < 3e-2
    assert abs(loss - lo) <= 3e-2 * lo
    gg = _unflat(g)
    for name in go:
        a, b = gg[name].ravel(), go[name].ravel()
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-20)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        print(f"  grad {name}: rel L2 {rel:.2e}, cosine {cos:.6f}")
        assert rel < 5e-2 and cos > 0.995, (name, rel, cos)


def test_predict_full_batch_matches_oracle():
    """640 leaves through lbm_surrogate_predict with two members and target mode 2: after the
    library's own base is removed, each member's output is the oracle's network output in
    standardised units, destandardised."""
    lbm = _lbm()
    n = 640
    leaves = _leaves_logk(n, 21)
    x = _inputs(n, 0, leaves)
    pa, pb = S.init_params(23), S.init_params(29)
    shift, scale, m0, s0, m1, s1 = -4.0, 1.3, 0.2, 0.7, -0.1, 0.9
    xn = x.copy()
    xn[:, :4] = (x[:, :4] - shift) / scale
    xn[:, 5:] = (x[:, 5:] - shift) / scale
    with lbm.Surrogate(2, 0) as sur:
        c, w = _base_from_predict(sur, x, 2, n_models=2)
        sur.set_params(0, _flat(pa))
        sur.set_params(1, _flat(pb))
        norm = np.array([shift, scale, m0, s0, m1, s1, -1e30, 1e30, -1e30, 1e30, -1e30, 1e30, 2], dtype=np.float32)
        sur.set_normalization(norm)
        pred = sur.predict(_t(x)).cpu().numpy().astype(np.float64)
    for k, pk in enumerate((pa, pb)):
        net, _ = S.forward(_unflat(_bf16(_flat(pk))), _bf16(xn).astype(np.float64))
        ref = np.stack([net[:, 0] * s0 + m0, net[:, 1] * s1 + m1], axis=1)
        got = (pred[k] - c) / w
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"member {k}: 640-leaf prediction rel L2 {err:.2e}")
        assert err < 3e-2


def _gate_setup(sur, n_models, seed):
    """Members that differ only in the head bias (so their spread is set by the per-leaf width w)."""
    p = S.init_params(seed)
    for m in range(n_models):
        q = {k: v.copy() for k, v in p.items()}
        q["bh"] = q["bh"] + 0.02 * np.array([m - 1.5, 0.7 * (1.5 - m)])
        sur.set_params(m, _flat(q))


def test_surrogate_keff_gate_matches_oracle():
    """lbm_surrogate_keff on the quadtree leaves of a 256^2 field with a per-size gate: each leaf's
    accept / fall-back decision and accepted K* against the oracle gate on the same member
    predictions and statistics (3 % and per-size spreads, statistic ranges that exclude some
    leaves); the fallback leaves' K* and status against lbm_local_keff_batch bit for bit."""
    import torch
    lbm = _lbm()
    kap = synth.lognormal_kappa(256, 256, 8.0, 1.5, seed=33).astype(np.float32)
    kt = _t(kap)
    lt = torch.from_numpy(synth.quadtree_leaves(256, 256, seed=33)).cuda()
    sizes = lt[:, 2].cpu().numpy()
    p = lbm.Params(nx=256, ny=256, tau=1.0, eps=1.0)
    with lbm.Surrogate(4, 0) as sur:
        _gate_setup(sur, 4, 37)
        x, st = lbm.lbm_patches(kt, lt)
        stn = st.cpu().numpy()
        lo = np.percentile(stn, 3, axis=0).astype(np.float32)
        hi = np.percentile(stn, 97, axis=0).astype(np.float32)
        norm = np.array([-4.6, 1.5, 0.0, 2.0, 0.0, 2.0, lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], 2], dtype=np.float32)
        sur.set_normalization(norm)
        pred = sur.predict(x).cpu().numpy()
        per_size = np.array([0.03, 0.03, 0.03, 0.05, 0.04, 0.03, 0.02], dtype=np.float32)
        sur.set_gate(per_size)
        # the library keeps the per-size limits in FP32: the oracle takes the same values
        gates = {"3pct": (0.03, 0.03), "per_size": (0.0, {1 << c: float(per_size[c]) for c in range(7)})}
        for name, (smax, ospread) in gates.items():
            acc_o, keff_o = S.gate(pred, stn, sizes, lo, hi, ospread)
            keff, fb, status, nfb, worst = sur.keff(p, kt, lt, spread_max=smax, g_const=1e-6, tol_rel=0.0,
                                                    max_steps=300)
            keff, fb, status = keff.cpu().numpy(), fb.cpu().numpy(), status.cpu().numpy()
            print(f"gate {name}: {acc_o.sum()} of {len(acc_o)} accepted by the oracle")
            assert 0 < acc_o.sum() < len(acc_o)
            np.testing.assert_array_equal(fb, (~acc_o).astype(np.int32))
            assert nfb == int((~acc_o).sum()) and worst == lbm.LBM_OK
            np.testing.assert_allclose(keff[acc_o], keff_o[acc_o], rtol=1e-15, atol=0)
            rej = np.nonzero(~acc_o)[0]
            ref_k, ref_s, _, _ = lbm.local_keff(p, kt, lt[torch.from_numpy(rej).cuda()].contiguous(), 1e-6, 0.0, 300, 64,
                                                True)
            np.testing.assert_array_equal(keff[rej], ref_k.cpu().numpy())
            np.testing.assert_array_equal(status[rej], ref_s.cpu().numpy())
            assert (status[acc_o] == 0).all()
        # a leaf size the path does not take (48) and a leaf outside the field are rejected
        for bad in ([[0, 0, 48]], [[240, 0, 32]]):
            with pytest.raises(lbm.LbmError) as ei:
                sur.keff(p, kt, torch.tensor(bad, dtype=torch.int32, device="cuda"), 0.03, 1e-6, 0.0, 10)
            assert ei.value.status == lbm.LBM_EINVAL


def test_gate_routes_blocks():
    """lbm_upscale with an ensemble: spread_max tiny sends every block to local LBM, and the result
    is then the LBM-only upscaling bit for bit; a generous gate accepts every in-range block and
    returns exp(ensemble mean) with zero off-diagonals."""
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
        pred = sur.predict(x).cpu().numpy().astype(np.float64)
    ks = k_sur.cpu().numpy().reshape(16, 4)
    np.testing.assert_allclose(ks[:, 0], np.exp(pred[:, :, 0].sum(axis=0) / 3), rtol=1e-15)
    np.testing.assert_allclose(ks[:, 3], np.exp(pred[:, :, 1].sum(axis=0) / 3), rtol=1e-15)
    assert (ks[:, 1] == 0).all() and (ks[:, 2] == 0).all()
