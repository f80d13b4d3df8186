"""The upscaled model in three dimensions on the GPU: coarse D3Q19 runs with a tensor K* per
cell (Eq. 18 in 3-D) and the block average, against the D3Q19 oracle's tensor mode."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _lbm():
    import paper_1312_0195_gb300 as lbm
    return lbm


def _tensor_field(shape, seed):
    rng = np.random.default_rng(seed)
    K = np.zeros(shape + (3, 3))
    for i in range(3):
        K[..., i, i] = 1e-2 * np.exp(0.8 * rng.standard_normal(shape))
    off = 1.5e-3 * rng.standard_normal(shape + (3, 3))
    off[..., [0, 1, 2], [0, 1, 2]] = 0.0
    return K + off


def _gpu_tensor_run(K, tau, nu, eps, g, steps, storage=0, block=1):
    """Coarse grid created from K (fine lattice units) and block, run `steps` steps."""
    import torch
    lbm = _lbm()
    nz, ny, nx = K.shape[:3]
    fine = lbm.Params3D(nx=nx * block, ny=ny * block, nz=nz * block, tau=tau, nu=nu, eps=eps, gx=g[0], gy=g[1],
                        gz=g[2], storage=storage)
    with lbm.Grid3D.coarse(fine, block, torch.from_numpy(np.ascontiguousarray(K)).cuda()) as G:
        G.step(steps)
        out = [t.cpu().numpy().astype(np.float64) for t in G.fields()]
        mean = np.array(G.mean_velocity())
        return out, mean, G.params


@pytest.mark.parametrize("storage", [0, 2])
def test_tensor_grid_matches_oracle(storage):
    """block = 1: the coarse parameters are the fine ones, so this is the tensor step itself."""
    K = _tensor_field((5, 6, 37), seed=91)
    tau, nu, eps, g, steps = 0.9, 0.08, 0.8, (1.2e-6, -0.8e-6, 0.5e-6), 150
    (r, u, v, w), mean, _ = _gpu_tensor_run(K, tau, nu, eps, g, steps, storage)
    p = oracle.Problem3D(tau, nu, eps, ktensor=K, g=g)
    f = p.rest()
    p.run(f, steps)
    ro, uo, vo, wo = p.fields(f)
    scale = max(np.abs(uo).max(), np.abs(vo).max(), np.abs(wo).max())
    tol = 1e-7 if storage == 2 else 1e-5          # fields come back as float32
    for a, b in ((u, uo), (v, vo), (w, wo)):
        np.testing.assert_allclose(a, b, rtol=0, atol=tol * scale)
    np.testing.assert_allclose(r, ro, rtol=0, atol=2.4e-7)
    np.testing.assert_allclose(mean, p.mean_velocity(f), rtol=0, atol=(1e-9 if storage == 2 else 1e-6) * scale)


def test_coarse_parameters_and_scaling():
    """block = 4: tau, nu, G and K* are rescaled (Section 3's coarse parameters); the run equals the
    oracle's run with the rescaled values."""
    lbm = _lbm()
    fine = lbm.Params3D(nx=16, ny=12, nz=8, tau=0.8, nu=0.1, eps=0.9, gx=1e-6, gy=-2e-6, gz=0.5e-6)
    c = lbm.lbm3d_coarse_params(fine, 4)
    assert (c.nx, c.ny, c.nz) == (4, 3, 2)
    assert abs(c.tau - (0.5 + 0.3 / 4)) < 1e-15 and abs(c.nu - 0.025) < 1e-15
    assert (c.gx, c.gy, c.gz) == (4e-6, -8e-6, 2e-6)
    K = _tensor_field((2, 3, 4), seed=92) * 16.0          # fine lattice units: coarse K* = K / 16
    (r, u, v, w), _, cp = _gpu_tensor_run(K, 0.8, 0.1, 0.9, (1e-6, -2e-6, 0.5e-6), 120, storage=2, block=4)
    p = oracle.Problem3D(c.tau, c.nu, c.eps, ktensor=K / 16.0, g=(c.gx, c.gy, c.gz))
    f = p.rest()
    p.run(f, 120)
    _, uo, vo, wo = p.fields(f)
    scale = max(np.abs(uo).max(), np.abs(vo).max(), np.abs(wo).max())
    for a, b in ((u, uo), (v, vo), (w, wo)):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-7 * scale)
    with pytest.raises(lbm.LbmError):
        lbm.lbm3d_coarse_params(fine, 5)


def test_diagonal_tensor_is_the_scalar_grid():
    import torch
    lbm = _lbm()
    k = synth.lognormal_kappa3d(8, 6, 10, 2.0, 1.5, seed=93)
    K = np.zeros(k.shape + (3, 3))
    for i in range(3):
        K[..., i, i] = k.astype(np.float64)
    g = (1e-6, 0.5e-6, -0.7e-6)
    (r, u, v, w), _, _ = _gpu_tensor_run(K, 0.7, 0.1, 1.0, g, 100)
    nz, ny, nx = k.shape
    p = lbm.Params3D(nx=nx, ny=ny, nz=nz, tau=0.7, nu=0.1, eps=1.0, gx=g[0], gy=g[1], gz=g[2])
    with lbm.Grid3D(p, torch.from_numpy(k).cuda()) as G:
        G.step(100)
        rs, us, vs, ws = (t.cpu().numpy().astype(np.float64) for t in G.fields())
    scale = max(np.abs(us).max(), np.abs(vs).max(), np.abs(ws).max())
    for a, b in ((u, us), (v, vs), (w, ws)):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * scale)


def test_block_average3_is_the_cube_mean():
    import torch
    lbm = _lbm()
    x = np.random.default_rng(94).standard_normal((12, 8, 20)).astype(np.float32)
    out = lbm.lbm3d_block_average(torch.from_numpy(x).cuda(), 4).cpu().numpy()
    ref = x.astype(np.float64).reshape(3, 4, 2, 4, 5, 4).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-6)
    with pytest.raises(lbm.LbmError):
        lbm.lbm3d_block_average(torch.from_numpy(x).cuda(), 3)


def test_singular_or_non_finite_tensor_rejected():
    import torch
    lbm = _lbm()
    fine = lbm.Params3D(nx=2, ny=2, nz=2, tau=1.0, eps=1.0, nu=0.1)
    K = np.zeros((2, 2, 2, 3, 3))
    K[..., 0, 0] = K[..., 1, 1] = K[..., 2, 2] = 1e-2
    K[1, 1, 1] = [[-0.05, 0, 0], [0, 1e-2, 0], [0, 0, 1e-2]]      # K + (eps nu / 2) I singular
    with pytest.raises(lbm.LbmError):
        lbm.Grid3D.coarse(fine, 1, torch.from_numpy(K).cuda())
    K[1, 1, 1] = np.nan
    with pytest.raises(lbm.LbmError):
        lbm.Grid3D.coarse(fine, 1, torch.from_numpy(K).cuda())


def test_upscaled_pipeline_small():
    """The whole method in 3-D on a 32^3 field, r = 8: local problems on the GPU give K* per
    block, the coarse run with those K* matches the oracle's coarse run, and the coarse velocity
    approximates the block-averaged fine velocity."""
    import torch
    lbm = _lbm()
    n, r = 32, 8
    kap = synth.lognormal_kappa3d(n, n, n, 4.0, 1.0, seed=95)
    kt = torch.from_numpy(kap).cuda()
    tau, g = 1.0, 1e-6
    leaves = torch.tensor([(x, y, z, r) for z in range(0, n, r) for y in range(0, n, r) for x in range(0, n, r)],
                          dtype=torch.int32, device="cuda")
    keff, st, _, _ = lbm.local_keff3(lbm.Params3D(nx=n, ny=n, nz=n, tau=tau, eps=1.0), kt, leaves, g, 1e-9, 200000,
                                     64)
    assert (st.cpu().numpy() == 0).all()
    kc = keff.reshape(n // r, n // r, n // r, 3, 3)
    fine = lbm.Params3D(nx=n, ny=n, nz=n, tau=tau, eps=1.0, gx=g)
    steps = 4000
    with lbm.Grid3D(fine, kt) as F:
        F.step(steps)
        _, uf, vf, wf = F.fields()
        avg = [lbm.lbm3d_block_average(t, r).cpu().numpy().astype(np.float64) for t in (uf, vf, wf)]
    with lbm.Grid3D.coarse(fine, r, kc) as Cg:
        Cg.step(steps // r)
        _, uc, vc, wc = (t.cpu().numpy().astype(np.float64) for t in Cg.fields())
        c = Cg.params
    p = oracle.Problem3D(c.tau, c.nu, c.eps, ktensor=kc.cpu().numpy() / (r * r), g=(c.gx, c.gy, c.gz))
    f = p.rest()
    p.run(f, steps // r)
    _, uo, vo, wo = p.fields(f)
    scale = np.abs(uo).max()
    for a, b in ((uc, uo), (vc, vo), (wc, wo)):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * scale)
    err = np.sqrt(sum(((a - b) ** 2).sum() for a, b in zip((uc, vc, wc), avg)) / sum((b ** 2).sum() for b in avg))
    assert err < 0.35, err


def test_upscale3_is_the_local_problem_per_block():
    """lbm3d_upscale: one cubic leaf per coarse cell, K* in the coarse grid's layout, the same
    values as the batched local problems on the same cubes (also with oversampling)."""
    import torch
    lbm = _lbm()
    n, r = 24, 8
    kap = torch.from_numpy(synth.lognormal_kappa3d(n, n, n, 3.0, 1.0, seed=96)).cuda()
    for m in (0, 2):
        p = lbm.Params3D(nx=n, ny=n, nz=n, tau=1.0, eps=1.0, margin=m)
        kc, nnc, st = lbm.lbm3d_upscale(p, kap, r, 1e-6, 0.0, 300)
        assert kc.shape == (3, 3, 3, 3, 3) and nnc == 0 and st == 0
        cubes = torch.tensor([(x, y, z, r) for z in range(0, n, r) for y in range(0, n, r) for x in range(0, n, r)],
                             dtype=torch.int32, device="cuda")
        ke, _, _, _ = lbm.local_keff3(p, kap, cubes, 1e-6, 0.0, 300, 64)
        np.testing.assert_array_equal(kc.reshape(-1, 3, 3).cpu().numpy(), ke.cpu().numpy())


@pytest.mark.parametrize("storage", [0, 2])
def test_tensor_layers_darcy_closed_form_on_gpu(storage):
    """The oracle pin's closed form on the GPU tensor grid: Darcy flow (tau = 1/2, E3's nu) through
    two-cell layers of a non-symmetric K*, driven along y; u_x constant, u_y and u_z from K_yx,
    K_zx and the layer pressure gradient."""
    ex = synth.paper_experiment("E3", ratio=10.0, ny=1)
    k1 = float(ex["kappa"][0, 0])
    tau, nu, eps, g = ex["tau"], ex["nu"], ex["eps"], 1e-6
    band = lambda *v: np.repeat(np.array(v), 2) * k1          # noqa: E731
    kxx, kyy = band(2, 4, 1, 3), band(1, 5, 2, 8)
    kxy, kyx, kzx = band(0.3, -0.5, 0.2, 0.4), band(-0.2, 0.6, 0.1, -0.3), band(0.1, 0.2, -0.1, 0.3)
    K = np.zeros((2, 2, kxx.size, 3, 3))
    K[..., 0, 0], K[..., 1, 1], K[..., 2, 2] = kxx, kyy, 3 * k1
    K[..., 0, 1], K[..., 1, 0], K[..., 2, 0] = kxy, kyx, kzx
    (r, u, v, w), _, _ = _gpu_tensor_run(K, tau, nu, eps, (0.0, g, 0.0), 8000, storage)
    c = g * np.sum(kxy / kxx) / (nu * np.sum(1.0 / kxx))
    dp = (kxy * g - nu * c) / kxx
    tol = 1e-5 if storage == 2 else 2e-3
    np.testing.assert_allclose(u[0, 0, :], c, rtol=tol)
    np.testing.assert_allclose(v[0, 0, :], (kyy * g - kyx * dp) / nu, rtol=tol)
    uz = -kzx * dp / nu
    np.testing.assert_allclose(w[0, 0, :], uz, rtol=0, atol=tol * np.abs(uz).max())
