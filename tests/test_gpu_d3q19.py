"""D3Q19 grids (Section 2's scheme in three dimensions) on the GPU against the D3Q19 oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _lbm():
    import paper_1312_0195_gb300 as lbm
    return lbm


def _field(nz, ny, nx, seed):
    rng = np.random.default_rng(seed)
    z = np.stack([synth.gaussian_random_field(nx, ny, 3.0, seed=seed * 100 + k) for k in range(nz)])
    z = 0.6 * z + 0.4 * rng.standard_normal((nz, ny, nx))
    return (1e-2 * np.exp(1.5 * z)).astype(np.float32)


def gpu3(kap, tau, nu, eps, g, steps, storage=0):
    import torch
    lbm = _lbm()
    nz, ny, nx = kap.shape
    p = lbm.Params3D(nx=nx, ny=ny, nz=nz, tau=tau, nu=nu, eps=eps, gx=g[0], gy=g[1], gz=g[2], storage=storage)
    with lbm.Grid3D(p, torch.from_numpy(np.ascontiguousarray(kap)).cuda()) as G:
        G.step(steps)
        out = [t.cpu().numpy().astype(np.float64) for t in G.fields()]
        mean = np.array(G.mean_velocity())
    return out, mean


def ora3(kap, tau, nu, eps, g, steps):
    p = oracle.Problem3D(tau, nu, eps, kappa=kap.astype(np.float64), g=g)
    f = p.rest()
    p.run(f, steps)
    return list(p.fields(f)), p.mean_velocity(f)


@pytest.mark.parametrize("shape", [(10, 12, 20), (7, 5, 131)])
def test_d3q19_fp32_matches_oracle(shape):
    kap = _field(*shape, seed=61)
    kap[1, 2, 3] = 0.0
    kap[2, 3, 4] = np.inf
    args = (kap, 0.8, 0.1, 0.9, (2e-6, -1e-6, 1.5e-6), 200)
    (r, u, v, w), mean = gpu3(*args)
    (ro, uo, vo, wo), mo = ora3(*args)
    scale = max(np.abs(uo).max(), np.abs(vo).max(), np.abs(wo).max())
    for a, b in ((u, uo), (v, vo), (w, wo)):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-5 * scale)
    np.testing.assert_allclose(r, ro, rtol=0, atol=2.4e-7)
    assert u[1, 2, 3] == 0.0 and v[1, 2, 3] == 0.0 and w[1, 2, 3] == 0.0
    np.testing.assert_allclose(mean, mo, rtol=2e-5, atol=1e-6 * scale)


def test_d3q19_fp64_matches_oracle_to_roundoff():
    kap = _field(6, 9, 11, seed=62)
    args = (kap, 0.7, 0.05, 0.8, (1e-6, 2e-6, -1e-6), 300)
    (r, u, v, w), mean = gpu3(*args, storage=2)
    (ro, uo, vo, wo), mo = ora3(*args)
    scale = max(np.abs(uo).max(), np.abs(vo).max(), np.abs(wo).max())
    for a, b in ((u, uo), (v, vo), (w, wo)):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-7 * scale)       # fields come back as float32
    np.testing.assert_allclose(mean, mo, rtol=1e-9, atol=1e-9 * scale)     # FP64 mean


def test_d3q19_full_size_sampled_against_oracle_windows():
    """256^3 (the benchmarked lattice, 16.8 M cells): after n steps a cell depends only on the
    cells within n of it, so periodic oracle windows of side 2 n + 9 reproduce sampled cells."""
    import torch
    lbm = _lbm()
    n, N = 6, 256
    rng = np.random.default_rng(63)
    kap = (1e-2 * np.exp(1.5 * rng.standard_normal((N, N, N)))).astype(np.float32)
    tau, nu, eps, g = 0.6, 0.2 / 6, 1.0, (1e-6, 0.0, 0.0)
    p = lbm.Params3D(nx=N, ny=N, nz=N, tau=tau, nu=nu, eps=eps, gx=g[0], gy=g[1], gz=g[2])
    pts = [tuple(int(v) for v in rng.integers(0, N, 3)) for _ in range(6)] + [(0, 0, 0), (N - 1, N - 1, N - 1)]
    with lbm.Grid3D(p, torch.from_numpy(kap).cuda()) as G:
        G.step(n)
        rho, u, v, w = G.fields()
        vals = [(float(u[z, y, x]), float(v[z, y, x]), float(w[z, y, x]), float(rho[z, y, x])) for (x, y, z) in pts]
    W = 2 * n + 9
    h = W // 2
    for (x, y, z), (ug, vg, wg, rg) in zip(pts, vals):
        zi = (np.arange(z - h, z - h + W) % N)[:, None, None]
        yi = (np.arange(y - h, y - h + W) % N)[None, :, None]
        xi = (np.arange(x - h, x - h + W) % N)[None, None, :]
        (ro, uo, vo, wo), _ = ora3(kap[zi, yi, xi], tau, nu, eps, g, n)
        s = max(abs(uo[h, h, h]), abs(vo[h, h, h]), abs(wo[h, h, h]), 1e-30)
        assert abs(ug - uo[h, h, h]) <= 1e-5 * s + 1e-13
        assert abs(vg - vo[h, h, h]) <= 1e-5 * s + 1e-13
        assert abs(wg - wo[h, h, h]) <= 1e-5 * s + 1e-13
        assert abs(rg - ro[h, h, h]) <= 2.4e-7


def test_d3q19_rejects_bad_input():
    import torch
    lbm = _lbm()
    kap = torch.full((4, 4, 4), 0.01, device="cuda")
    kap[1, 1, 1] = float("nan")
    with pytest.raises(lbm.LbmError):
        lbm.Grid3D(lbm.Params3D(nx=4, ny=4, nz=4, tau=1.0), kap)
    with pytest.raises(lbm.LbmError):
        lbm.Grid3D(lbm.Params3D(nx=4, ny=4, nz=4, tau=0.4), torch.full((4, 4, 4), 0.01, device="cuda"))
