"""GPU local-global local problems (lbm_local_keff_lg) against the oracle (orc_local_lg).

Inputs on both sides are the same: the field, and coarse (rho - 1, u, v) arrays per drive that
the GPU interpolates to the patch itself while the oracle takes them through
oracle.coarse_to_fine. The GPU stores FP32 deviations and reduces window means in FP64."""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _lbm():
    import paper_1312_0195_gb300 as lbm
    return lbm


def _coarse_state(nbx, nby, seed, g, eps, kap_scale, nu):
    """Smooth, seeded coarse states of the size a coarse run gives: rho - 1 ~ 3 eps G x (a few
    cells), velocities ~ kappa G / nu."""
    rng = np.random.default_rng(seed)
    out = np.empty((2, 3, nby, nbx), dtype=np.float32)
    jj, ii = np.meshgrid(np.arange(nby), np.arange(nbx), indexing="ij")
    for d in range(2):
        ph = rng.uniform(0, 2 * np.pi, 3)
        out[d, 0] = 3 * eps * g * 8 * (np.sin(2 * np.pi * ii / nbx + ph[0]) + 0.5 * np.cos(2 * np.pi * jj / nby + ph[1]))
        u = kap_scale * g / nu * (1.0 + 0.3 * np.sin(2 * np.pi * (ii + jj) / nbx + ph[2]))
        out[d, 1] = u if d == 0 else 0.2 * u
        out[d, 2] = 0.2 * u if d == 0 else u
    return out


def _run_gpu(kap, block, margin, coarse, tau, nu, eps, g, tol, max_steps, ring=2, fallback=None, storage=0, warm=0):
    import torch
    lbm = _lbm()
    ny, nx = kap.shape
    p = lbm.Params(nx=nx, ny=ny, tau=tau, nu=nu, eps=eps, margin=margin, storage=storage, warm_start=warm)
    kt = torch.from_numpy(np.ascontiguousarray(kap, dtype=np.float32)).cuda()
    ct = torch.from_numpy(np.ascontiguousarray(coarse, dtype=np.float32)).cuda()
    fb = None if fallback is None else torch.from_numpy(np.ascontiguousarray(fallback, dtype=np.float64)).cuda()
    ke, st, steps, win, worst, nfb = lbm.local_keff_lg(p, kt, block, ct, g, tol, max_steps, ring=ring, fallback=fb)
    out = (ke.cpu().numpy(), st.cpu().numpy(), steps.cpu().numpy(), win.cpu().numpy(), worst)
    return out if fallback is None else out + (nfb,)


def _run_oracle(kap, block, margin, coarse, bx, by, tau, nu, eps, g, tol, max_steps, ring=2, warm=False):
    ny, nx = kap.shape
    se = block + 2 * margin
    x0, y0 = bx * block - margin, by * block - margin
    xs, ys = (x0 + np.arange(se)) % nx, (y0 + np.arange(se)) % ny
    k = np.asarray(kap, dtype=np.float32)[np.ix_(ys, xs)].astype(np.float64)
    st = np.stack([oracle.coarse_to_fine(coarse[d].astype(np.float64), block, x0, y0, se).transpose(1, 2, 0)
                   for d in range(2)])
    for d in range(2):
        st[d, ..., 0] -= float(coarse[d, 0, by, bx])                # the block's own coarse density
    if warm:
        st = oracle.lg_darcy_state(k, st, nu, eps, g)
    return oracle.local_keff_lg(k, margin, st, tau, nu, eps, g, tol=tol, max_steps=max_steps, ring=ring)


@pytest.mark.parametrize("ring", [1, 2])
def test_fixed_steps_match_oracle(ring):
    """A log-normal field (sigma 1.5), 16-cell blocks grown by 4, a smooth coarse state, 384 fixed
    steps (the pressure-only ring refreshed at five checks): every block's window means (u, v and
    the density gradient, per drive) and K* match the oracle to 1e-4 of their scales, tau = 1 and
    tau = 0.8."""
    kap = synth.lognormal_kappa(64, 64, 6.0, 1.5, seed=41)
    eps, g = 0.9, 1e-6
    for tau in (1.0, 0.8):
        nu = (tau - 0.5) / 3.0
        coarse = _coarse_state(4, 4, 7, g, eps, 1e-2, nu)
        ke, st, steps, win, worst = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 0.0, 384, ring=ring)
        assert worst == 0 and (steps == 384).all()
        for by in range(4):
            for bx in range(4):
                ref = _run_oracle(kap, 16, 4, coarse, bx, by, tau, nu, eps, g, 0.0, 384, ring=ring)
                w, wr = win[by, bx], ref["window"]
                for d in range(2):
                    us = np.hypot(*wr[d, :2])
                    gs = np.hypot(*wr[d, 2:]) + 3 * eps * g
                    assert np.abs(w[d, :2] - wr[d, :2]).max() <= 1e-4 * us, (tau, bx, by, d, w[d], wr[d])
                    assert np.abs(w[d, 2:] - wr[d, 2:]).max() <= 1e-4 * gs, (tau, bx, by, d, w[d], wr[d])
                k, kr = ke[by, bx], ref["keff"]
                scale = np.sqrt(abs(kr[0] * kr[3]))
                assert np.abs(k - kr).max() <= 1e-4 * scale, (tau, bx, by, k, kr)


@pytest.mark.parametrize("ring", [1, 2])
def test_tolerance_stop_matches_oracle(ring):
    """The same set-up at tol 1e-8 (stop on the whole window velocity vector): K* agrees with the
    oracle's within the stop test's band, 1e-3 of the tensor's scale."""
    kap = synth.lognormal_kappa(64, 64, 6.0, 1.5, seed=43)
    tau, eps, g = 1.0, 1.0, 1e-6
    nu = (tau - 0.5) / 3.0
    coarse = _coarse_state(4, 4, 9, g, eps, 1e-2, nu)
    ke, st, steps, win, worst = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 1e-8, 200000, ring=ring)
    assert worst == 0
    for by in range(4):
        for bx in range(4):
            ref = _run_oracle(kap, 16, 4, coarse, bx, by, tau, nu, eps, g, 1e-8, 200000, ring=ring)
            kr = ref["keff"]
            scale = np.sqrt(abs(kr[0] * kr[3]))
            assert np.abs(ke[by, bx] - kr).max() <= 1e-3 * scale, (bx, by, ke[by, bx], kr)


@pytest.mark.parametrize("ring", [1, 2])
def test_uniform_medium_under_a_linear_state_gives_kappa(ring):
    """A uniform medium whose coarse state is a linear pressure field with the matching Darcy
    velocity (bilinear interpolation reproduces it exactly away from the periodic wrap): every
    block whose grown patch does not wrap gets K* = kappa I in FP32 (1e-4), although the
    window's mean force is far from G I."""
    kap0, tau, eps, g, block, margin = 0.02, 1.0, 0.9, 1e-6, 16, 4
    nu = (tau - 0.5) / 3.0
    nb = 8
    # a uniform medium up to a 1e-6 relative ripple, so that the patches are not skipped as uniform
    kap = (kap0 * (1.0 + 1e-6 * (np.indices((nb * block, nb * block)).sum(axis=0) % 2))).astype(np.float32)
    X = (np.arange(nb) + 0.5) * block - 0.5 - nb * block / 2           # coarse centres in fine units
    Xc, Yc = np.meshgrid(X, X)
    coarse = np.empty((2, 3, nb, nb), dtype=np.float32)
    for d, (a, b) in enumerate([(0.3, 0.2), (-0.1, 0.4)]):
        coarse[d, 0] = 3 * eps * g * (a * Xc + b * Yc)
        coarse[d, 1] = kap0 / nu * ((g if d == 0 else 0.0) - g * a)
        coarse[d, 2] = kap0 / nu * ((g if d == 1 else 0.0) - g * b)
    ke, st, steps, win, worst = _run_gpu(kap, block, margin, coarse, tau, nu, eps, g, 1e-9, 200000, ring=ring)
    inner = ke[1:nb - 1, 1:nb - 1].reshape(-1, 4) / kap0
    np.testing.assert_allclose(inner, np.tile([1.0, 0.0, 0.0, 1.0], (len(inner), 1)), rtol=0, atol=1e-4)
    np.testing.assert_allclose(win[2, 3, 0, 2:] / (3 * eps * g), [0.3, 0.2], rtol=1e-4)


def test_rejections():
    import torch
    lbm = _lbm()
    kap = torch.full((32, 32), 0.01, device="cuda")
    coarse = torch.zeros((2, 3, 2, 2), device="cuda")
    for kw in (dict(margin=1), dict(margin=25), dict(margin=15, storage=2)):
        p = lbm.Params(nx=32, ny=32, tau=1.0, **kw)
        with pytest.raises(lbm.LbmError) as ei:
            lbm.local_keff_lg(p, kap, 16, coarse, 1e-6, 1e-8, 100)
        assert ei.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.local_keff_lg(lbm.Params(nx=32, ny=32, tau=1.0, margin=4), kap, 16, coarse.cpu(), 1e-6, 1e-8, 100)


def test_fallback_selection_matches_the_oracle_rule():
    """With fallback tensors the library keeps a block's K* (symmetrised) only when it converged,
    is positive definite after symmetrising and its force matrix has condition number <= 10:
    the kept/fallen-back blocks and every output tensor equal oracle.lg_select applied to the
    library's own raw K*, windows and statuses (both decide in FP64 from the same numbers)."""
    kap = synth.lognormal_kappa(128, 128, 6.0, 2.5, seed=45)
    tau, eps, g = 1.0, 1.0, 1e-6
    nu = (tau - 0.5) / 3.0
    coarse = _coarse_state(8, 8, 11, g, eps, 1e-2, nu)
    coarse[:, 0] *= 20.0                                   # strong pressure gradients: some F ill-conditioned
    raw, st, steps, win, worst = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 1e-8, 20000)
    ref = np.tile(np.array([1.0, 0.0, 0.0, 2.0]), (8, 8, 1))
    ke, st2, _, win2, _, nfb = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 1e-8, 20000, fallback=ref)
    np.testing.assert_array_equal(win2, win)               # the same runs, bit for bit
    exp, fb = oracle.lg_select(raw.reshape(-1, 4), win.reshape(-1, 2, 4), st.reshape(-1) == 0, ref.reshape(-1, 4),
                               g, eps)
    assert nfb == int(fb.sum()) and 0 < nfb < 64
    np.testing.assert_allclose(ke.reshape(-1, 4), exp, rtol=1e-14, atol=0)


def test_uniform_patches_run_no_local_problem():
    """A uniform field with one heterogeneous 16-cell square: blocks whose grown patch misses the
    square are uniform and get K* = kappa I exactly with 0 steps and a NaN window; the others run
    their local problems."""
    kap0, tau, eps, g, block, margin = 0.02, 1.0, 1.0, 1e-6, 16, 4
    nu = (tau - 0.5) / 3.0
    kap = np.full((128, 128), kap0, dtype=np.float32)
    kap[48:64, 48:64] = synth.lognormal_kappa(16, 16, 3.0, 1.0, seed=3)
    coarse = _coarse_state(8, 8, 5, g, eps, kap0, nu)
    ke, st, steps, win, worst = _run_gpu(kap, block, margin, coarse, tau, nu, eps, g, 1e-8, 200000)
    hetero = np.zeros((8, 8), dtype=bool)
    hetero[2:5, 2:5] = True                        # blocks whose patch (grown by 4) reaches 48..63
    assert (steps[~hetero] == 0).all() and np.isnan(win[~hetero]).all()
    np.testing.assert_array_equal(ke[~hetero], np.tile([kap0, 0.0, 0.0, kap0], ((~hetero).sum(), 1)).astype(np.float32).astype(np.float64))
    assert (steps[hetero] > 0).all() and (st == 0).all()


@pytest.mark.parametrize("ring", [1, 2])
def test_fp64_matches_oracle_to_roundoff(ring):
    """storage = LBM_F64 runs the local-global problems in FP64 (patches up to 45 cells): at 384
    fixed steps every window mean and K* matches the FP64 oracle to 1e-8 of its scale (the oracle
    stores full distributions of ~0.1 for velocities of ~4e-8: its own rounding is ~1e-9 of them)."""
    kap = synth.lognormal_kappa(64, 64, 6.0, 1.5, seed=47)
    tau, eps, g = 0.8, 0.9, 1e-6
    nu = (tau - 0.5) / 3.0
    coarse = _coarse_state(4, 4, 13, g, eps, 1e-2, nu)
    ke, st, steps, win, worst = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 0.0, 384, ring=ring, storage=2)
    assert worst == 0 and (steps == 384).all()
    for by in range(4):
        for bx in range(4):
            ref = _run_oracle(kap, 16, 4, coarse, bx, by, tau, nu, eps, g, 0.0, 384, ring=ring)
            w, wr = win[by, bx], ref["window"]
            for d in range(2):
                us = np.hypot(*wr[d, :2])
                gs = np.hypot(*wr[d, 2:]) + 3 * eps * g
                assert np.abs(w[d, :2] - wr[d, :2]).max() <= 1e-8 * us, (bx, by, d, w[d], wr[d])
                assert np.abs(w[d, 2:] - wr[d, 2:]).max() <= 1e-8 * gs, (bx, by, d, w[d], wr[d])
            kr = ref["keff"]
            assert np.abs(ke[by, bx] - kr).max() <= 1e-8 * np.sqrt(abs(kr[0] * kr[3]))


def test_darcy_start_matches_oracle():
    """warm_start = 1: the inner cells start from the Darcy flow with the ring's pressures held
    (CG to 1e-5 in shared memory; the oracle solves it directly). At 256 fixed steps the window
    means and K* match the oracle's runs from oracle.lg_darcy_state to 1e-4; at tol 1e-8 the
    Darcy-started runs take fewer steps than the runs from the coarse state and their window means
    agree within the stop test's band (median 1e-4, 90 % within 2e-3). In FP64 (the oracle) every
    block of this case lands within 8e-5 of a tol 1e-11 solve from either start; in FP32 one of
    the 32 runs, a block with little flow, stops far from its counterpart, so the bound is on the
    distribution."""
    kap = synth.lognormal_kappa(64, 64, 6.0, 2.0, seed=49)
    tau, eps, g = 1.0, 1.0, 1e-6
    nu = (tau - 0.5) / 3.0
    coarse = _coarse_state(4, 4, 15, g, eps, 1e-2, nu)
    ke, st, steps, win, worst = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 0.0, 256, warm=1)
    assert worst == 0
    for by in range(4):
        for bx in range(4):
            ref = _run_oracle(kap, 16, 4, coarse, bx, by, tau, nu, eps, g, 0.0, 256, warm=True)
            w, wr = win[by, bx], ref["window"]
            for d in range(2):
                us = np.hypot(*wr[d, :2])
                gs = np.hypot(*wr[d, 2:]) + 3 * eps * g
                assert np.abs(w[d, :2] - wr[d, :2]).max() <= 1e-4 * us, (bx, by, d, w[d], wr[d])
                assert np.abs(w[d, 2:] - wr[d, 2:]).max() <= 1e-4 * gs, (bx, by, d, w[d], wr[d])
    kw, sw, nw, ww, _ = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 1e-8, 200000, warm=1)
    kc, sc, nc, wc, _ = _run_gpu(kap, 16, 4, coarse, tau, nu, eps, g, 1e-8, 200000)
    assert (sw == 0).all() and (sc == 0).all()
    assert nw.sum() < nc.sum()
    # compare the window means (K* = nu U F^-1 amplifies their differences where F is nearly
    # singular, which is what the fallback rule guards against)
    # (blocks of the low-permeability phase carry ~1e-3 of the largest flow; their FP32 velocities
    # are compared on that field-wide scale)
    us = np.hypot(wc[..., 0], wc[..., 1])
    us = us + 1e-3 * us.max()
    gs = np.hypot(wc[..., 2], wc[..., 3]) + 3 * eps * g
    du = np.abs(ww[..., :2] - wc[..., :2]).max(axis=-1) / us
    dg = np.abs(ww[..., 2:] - wc[..., 2:]).max(axis=-1) / gs
    print(f"\nwindow differences: velocity median {np.median(du):.1e} p90 {np.percentile(du, 90):.1e} "
          f"max {du.max():.1e}; gradient median {np.median(dg):.1e} max {dg.max():.1e}")
    assert np.median(du) <= 1e-4 and np.percentile(du, 90) <= 2e-3
    assert np.median(dg) <= 1e-4 and np.percentile(dg, 90) <= 2e-3


def test_upscale_lg_is_the_sequence_of_its_calls():
    """lbm_upscale_lg equals, bit for bit, the calls it stands for: lbm_upscale (periodic, margin 0),
    two steady coarse runs (G along x, then y) with that K*, and lbm_local_keff_lg from their
    (rho - 1, u, v) with the periodic K* as fallback; passes = 0 returns the periodic K*."""
    import torch
    lbm = _lbm()
    n, r = 256, 16
    nb = n // r
    kt = torch.from_numpy(synth.channel_kappa(n, n, seed=5)).cuda()
    p = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, margin=4, warm_start=1)
    kw = dict(g_const=1e-6, tol_rel=1e-8, max_steps=30000, coarse_max_steps=20000, coarse_tol=1e-7)
    k1 = torch.empty((nb, nb, 4), dtype=torch.float64, device="cuda")
    st1, nfb1 = lbm.lbm_upscale_lg(p, kt, r, k1, passes=1, **kw)
    kp = torch.empty_like(k1)
    lbm.lbm_upscale(lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0), kt, r, kp, 1e-6, 1e-8, 30000)
    k0 = torch.empty_like(k1)
    lbm.lbm_upscale_lg(p, kt, r, k0, passes=0, **kw)
    assert torch.equal(k0, kp)
    cs = torch.empty((2, 3, nb, nb), dtype=torch.float32, device="cuda")
    for d in range(2):
        pd = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, gx=1e-6 if d == 0 else 0.0, gy=1e-6 if d == 1 else 0.0)
        lbm.lbm_coarse_run(pd, r, kp, None, 20000, 1e-7, 64, cs[d, 0], cs[d, 1], cs[d, 2])
        cs[d, 0] -= 1.0
    k2, st2, _, _, _, nfb2 = lbm.local_keff_lg(p, kt, r, cs, 1e-6, 1e-8, 30000, fallback=kp)
    assert torch.equal(k1, k2) and nfb1 == nfb2
    assert 0 < nfb1 < nb * nb
