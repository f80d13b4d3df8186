"""GPU parity of the fused step (liblbm.so through the C ABI) against the FP64 oracle.

Tolerances. The FP32 path must reach 1e-4 relative L2 on steady velocity.
Element-wise checks early in a run use |gpu - oracle| <= 1e-5 max|u|:
FP32 deviation storage rounds each population to ~6e-8 of its own size and a
cell's velocity sums nine of them, so a few hundred steps stay far below that.
FP64 storage must agree to ~1e-11 (only summation order differs). FP16 storage
(11-bit mantissa) has a fixed, deterministic error on its test case, measured on
a GB300 at 2.08e-2 (periodic) and 2.13e-2 (walls) relative L2; the test holds it
to 10 % above those values, so a change that makes FP16 storage worse fails.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _lbm():
    import paper_1312_0195_gb300 as lbm
    return lbm


def gpu_run(kap, tau, nu, eps, g, walls, steps, storage=0, check=0, gfield=None, scale=0.0):
    import torch
    lbm = _lbm()
    ny, nx = kap.shape
    p = lbm.Params(nx=nx, ny=ny, tau=tau, nu=nu, eps=eps, gx=g[0], gy=g[1],
                   bc=lbm.LBM_BC_WALLS_Y if walls else lbm.LBM_BC_PERIODIC, storage=storage, scale=scale)
    kt = torch.from_numpy(np.ascontiguousarray(kap, dtype=np.float32)).cuda()
    gt = None if gfield is None else torch.from_numpy(np.ascontiguousarray(gfield, dtype=np.float32)).cuda()
    with lbm.Grid(p, kt, gt) as G:
        n, resid, _ = G.step(steps, 0.0, check)
        assert n == steps
        rho, u, v = (t.cpu().numpy().astype(np.float64) for t in G.fields())
        mean = np.array(G.mean_velocity())
    return dict(rho=rho, u=u, v=v, mean=mean, resid=resid)


def oracle_run(kap, tau, nu, eps, g, walls, steps, check=0, gfield=None):
    k64 = np.asarray(kap, dtype=np.float32).astype(np.float64)     # same input values as the GPU
    gf = None if gfield is None else np.asarray(gfield, dtype=np.float32).astype(np.float64)
    p = oracle.Problem(tau, nu, eps, kappa=k64, g=g, gfield=gf, walls=walls)
    f = p.rest()
    _, resid, _ = p.run(f, steps, 0.0, check)
    rho, u, v = p.fields(f)
    return dict(rho=rho, u=u, v=v, mean=p.mean_velocity(f), resid=resid)


def rel_l2(a, b, ref=None):
    ref = b if ref is None else ref
    return np.linalg.norm(a - b) / np.linalg.norm(ref)


# ------------------------------------------------------------------ the 128x64 walled channel

def test_channel_128x64_steady_parity():
    """128x64, walls in y, tau = 1, eps = 1, nu = nu_eff, G = (1e-6, 0), log-normal K (ell = 8, sigma = 1).

    Both sides run the same 20000 steps (the step limit of the configuration; see the
    stop-rule reading) and are compared at that step count.
    """
    kap = synth.lognormal_kappa(128, 64, 8.0, 1.0, seed=1)
    nu = (1.0 - 0.5) / 3.0
    args = (kap, 1.0, nu, 1.0, (1e-6, 0.0), True, 20000)
    a = gpu_run(*args, check=64)
    b = oracle_run(*args, check=64)
    assert rel_l2(a["u"], b["u"]) < 1e-4
    assert np.linalg.norm(a["v"] - b["v"]) / np.linalg.norm(b["u"]) < 1e-4
    # rho is returned as float32: near 1.0 that resolves 6e-8, so compare to 2 ulps
    assert np.abs(a["rho"] - b["rho"]).max() <= 2.4e-7
    # domain K_eff from the mean flux, Eq. 17 applied to the whole channel
    k_gpu = nu * a["mean"][0] / 1e-6
    k_orc = nu * b["mean"][0] / 1e-6
    assert abs(k_gpu - k_orc) <= 1e-4 * abs(k_orc)
    # the residual is defined identically on both sides (FP32 vs FP64 noise allowed)
    assert a["resid"] > 0 and b["resid"] > 0


# ------------------------------------------------- tiles, ragged tails, edges

SHAPES = [(132, 68, False), (132, 68, True), (130, 66, True), (97, 35, False), (1, 16, True),
          (8, 1, False), (1, 1, False), (520, 3, True)]


@pytest.mark.parametrize("nx,ny,walls", SHAPES, ids=lambda v: str(v))
def test_fp32_elementwise_parity(nx, ny, walls):
    kap = synth.lognormal_kappa(nx, ny, 4.0, 1.5, seed=nx * 1000 + ny) if nx * ny > 1 else np.full((1, 1), 0.02)
    args = (kap, 0.8, 0.05, 0.9, (2e-6, -7e-7), walls, 300)
    a = gpu_run(*args)
    b = oracle_run(*args)
    scale = max(np.abs(b["u"]).max(), np.abs(b["v"]).max())
    assert np.abs(a["u"] - b["u"]).max() <= 1e-5 * scale
    assert np.abs(a["v"] - b["v"]).max() <= 1e-5 * scale
    assert np.abs(a["rho"] - b["rho"]).max() <= 1e-6


def test_guo_force_model_matches_oracle_guo_and_simplified():
    """Guo scheme (Section 2.1) on the GPU against the oracle's Guo scheme; and, as the paper's E1
    comparison shows and the algebra of the linear equilibrium implies, against the simplified scheme."""
    import torch
    lbm = _lbm()
    ex = synth.paper_experiment("E1")
    kap = ex["kappa"].astype(np.float32)
    outs = {}
    for storage in (0, 2):
        for fm in (0, 1):
            p = lbm.Params(nx=100, ny=100, tau=ex["tau"], nu=ex["nu"], eps=ex["eps"], gx=ex["g"][0],
                           storage=storage, force_model=fm)
            with lbm.Grid(p, torch.from_numpy(kap).cuda()) as G:
                G.step(1000, 0.0, 0)
                outs[storage, fm] = G.fields()[1].cpu().numpy().astype(np.float64)
    prob = oracle.Problem(ex["tau"], ex["nu"], ex["eps"], kappa=kap.astype(np.float64), g=ex["g"], guo=True)
    f = prob.rest()
    prob.run(f, 1000)
    _, uo, _ = prob.fields(f)
    scale = np.abs(uo).max()
    # FP64 storage: both schemes agree with the oracle's Guo run to the FP32 rounding of the returned field
    assert np.abs(outs[2, 1] - uo).max() <= 2e-7 * scale
    assert np.abs(outs[2, 0] - uo).max() <= 2e-7 * scale
    # FP32 storage: E1's drag is weak (1 - d ~ 1e-4), so rounding of the stored momentum is damped
    # slowly and drifts by up to ~6e-5 of max|u| over 1000 steps, in either scheme
    assert np.abs(outs[0, 1] - uo).max() <= 2e-4 * scale
    assert np.abs(outs[0, 0] - uo).max() <= 2e-4 * scale


def test_fp64_storage_matches_to_roundoff():
    kap = synth.lognormal_kappa(66, 40, 5.0, 2.0, seed=4)
    args = (kap, 0.7, 0.1, 0.8, (3e-6, 1e-6), True, 400)
    a = gpu_run(*args, storage=2)
    b = oracle_run(*args)
    scale = np.abs(b["u"]).max()
    assert np.abs(a["u"] - b["u"]).max() <= 1e-7 * scale      # fields are returned as float32
    np.testing.assert_allclose(a["mean"], b["mean"], rtol=1e-11, atol=1e-22)


@pytest.mark.parametrize("walls", [False, True])
def test_fp16_storage_error_is_bounded(walls):
    """FP16 storage keeps 11 significant bits per population. In this Darcy-like regime
    the density deviations are ~500x the velocity (grad p ~ eps nu u / kappa), and they
    sit in every population, so u is resolved to ~2 %: measured 2.081e-2 periodic and
    2.128e-2 with walls (3000 steps), bounded at 10 % above each."""
    kap = synth.lognormal_kappa(128, 64, 8.0, 1.0, seed=11)
    args = (kap, 1.0, 1.0 / 6.0, 1.0, (1e-6, 0.0), walls, 3000)
    a = gpu_run(*args, storage=1)
    b = oracle_run(*args)
    err = rel_l2(a["u"], b["u"])
    print(f"FP16 storage rel L2 error on u: {err:.3e}")
    measured = 2.128e-2 if walls else 2.081e-2          # GB300, this case, bit-reproducible
    assert err < 1.1 * measured


def test_residual_definition_matches_oracle():
    kap = synth.lognormal_kappa(64, 32, 6.0, 1.0, seed=5)
    args = (kap, 0.9, 0.05, 1.0, (1e-4, 0.0), False, 160)
    a = gpu_run(*args, check=16, storage=2)
    b = oracle_run(*args, check=16)
    assert abs(a["resid"] - b["resid"]) <= 1e-8 * b["resid"]
    a32 = gpu_run(*args, check=16)
    assert abs(a32["resid"] - b["resid"]) <= 1e-2 * b["resid"]


def test_force_field_parity():
    """Per-cell body force G(x) (the sinusoidal drive of Section 4.3)."""
    kap = synth.lognormal_kappa(80, 60, 6.0, 1.0, seed=6)
    gf = synth.sinusoidal_g_field(60, 1e-6)[:, :, :60]
    gf = np.concatenate([gf, gf[:, :, :20]], axis=2)
    args = (kap, 0.9, 0.05, 0.8, (0.0, 0.0), False, 400)
    a = gpu_run(*args, gfield=gf)
    b = oracle_run(*args, gfield=gf)
    scale = max(np.abs(b["u"]).max(), np.abs(b["v"]).max())
    assert np.abs(a["u"] - b["u"]).max() <= 1e-5 * scale
    assert np.abs(a["v"] - b["v"]).max() <= 1e-5 * scale


def test_infinite_and_zero_permeability():
    """kappa = +inf (no drag, plane Poiseuille) and kappa = 0 (blocked cells: u = 0)."""
    kap = np.full((32, 8), np.inf)
    kap[10:14, 2:5] = 0.0
    args = (kap, 1.0, 1.0 / 6.0, 1.0, (1e-6, 0.0), True, 2000)
    a = gpu_run(*args)
    b = oracle_run(*args)
    assert rel_l2(a["u"], b["u"]) < 1e-5
    assert np.abs(a["u"][10:14, 2:5]).max() == 0.0


# ------------------------------------------------------- full size, sampled

def test_full_size_4096_sampled_against_oracle_windows():
    """4096^2 periodic, log-normal K (sigma 2, ell 32, seed 2), tau = 0.6, in the bench's launch shape.

    After n steps a cell depends only on inputs within n cells, so the oracle run
    on a periodic window of side >= 2n + 1 centred on a cell gives that cell exactly.
    """
    import torch
    lbm = _lbm()
    n = 12
    N = 4096
    kap = synth.lognormal_kappa(N, N, 32.0, 2.0, seed=2).astype(np.float32)
    tau, nu, eps, g = 0.6, 0.1 / 3.0, 1.0, (1e-6, 0.0)
    p = lbm.Params(nx=N, ny=N, tau=tau, nu=nu, eps=eps, gx=g[0], gy=g[1])
    with lbm.Grid(p, torch.from_numpy(kap).cuda()) as G:
        G.step(n, 0.0, 0)
        rho, u, v = G.fields()
        rho, u, v = rho.cpu().numpy(), u.cpu().numpy(), v.cpu().numpy()
        # mass: the sum of all stored deviations (= sum of drho) stays at its initial 0
        state = torch.empty(lbm.lbm_grid_state_bytes(G.handle), dtype=torch.uint8, device="cuda")
        lbm.lbm_grid_save_state(G.handle, state)
        hdr = lbm.CKPT_HEADER_BYTES
        cur = state[hdr: hdr + (state.numel() - hdr) // 2].view(torch.float32)
        total_drho = float(cur.double().sum())
    rng = np.random.default_rng(0)
    pts = [(0, 0), (N - 1, N - 1), (0, N - 1), (N - 1, 0)] + [tuple(rng.integers(0, N, 2)) for _ in range(12)]
    W = 2 * n + 9
    h = W // 2
    for (x, y) in pts:
        win = synth.crop_periodic(kap, x - h, y - h, W, W).astype(np.float64)
        pr = oracle.Problem(tau, nu, eps, kappa=win, g=g)
        f = pr.rest()
        pr.run(f, n)
        ro, uo, vo = pr.fields(f)
        scale = max(abs(uo[h, h]), abs(vo[h, h]), 1e-30)
        assert abs(u[y, x] - uo[h, h]) <= 1e-5 * scale + 1e-12
        assert abs(v[y, x] - vo[h, h]) <= 1e-5 * max(scale, abs(vo[h, h])) + 1e-12
        assert abs(rho[y, x] - ro[h, h]) <= 1e-6
    # mass is conserved at full size up to FP32 rounding of the deviations (~1e-13 each)
    assert abs(total_drho) / (N * N) < 1e-14


def test_full_size_16384_channelised_sampled():
    """16384^2 channelised field (seed 5, contrast 1e4, eps 1, tau 1, G = (1e-6, 0)): the largest
    fine lattice of the workloads (19.3 GB of FP32 state), sampled against oracle windows after
    n steps, plus mass conservation on the raw state."""
    import torch
    lbm = _lbm()
    n = 8
    N = 16384
    kap = synth.channel_kappa(N, N, seed=5)
    tau, nu, eps, g = 1.0, 1.0 / 6.0, 1.0, (1e-6, 0.0)
    p = lbm.Params(nx=N, ny=N, tau=tau, nu=nu, eps=eps, gx=g[0], gy=g[1])
    kt = torch.from_numpy(kap).cuda()
    rng = np.random.default_rng(3)
    # half the samples on channel cells, half anywhere
    ys, xs = np.nonzero(kap[::97, ::89] > 1e-3)
    chan = [(int(xs[i] * 89), int(ys[i] * 97)) for i in rng.choice(len(xs), 6, replace=False)]
    pts = chan + [tuple(int(v) for v in rng.integers(0, N, 2)) for _ in range(6)] + [(0, 0), (N - 1, N - 1)]
    with lbm.Grid(p, kt) as G:
        del kt
        G.step(n, 0.0, 0)
        rho, u, v = G.fields()
        vals = [(float(u[y, x]), float(v[y, x]), float(rho[y, x])) for (x, y) in pts]
        del rho, u, v
        full = torch.empty(lbm.lbm_grid_state_bytes(G.handle), dtype=torch.uint8, device="cuda")
        lbm.lbm_grid_save_state(G.handle, full)
        hdr = lbm.CKPT_HEADER_BYTES
        total_drho = float(full[hdr: hdr + (full.numel() - hdr) // 2].view(torch.float32).sum(dtype=torch.float64))
        del full
    W = 2 * n + 9
    h = W // 2
    ref = []
    for (x, y) in pts:
        win = synth.crop_periodic(kap, x - h, y - h, W, W).astype(np.float64)
        pr = oracle.Problem(tau, nu, eps, kappa=win, g=g)
        f = pr.rest()
        pr.run(f, n)
        ro, uo, vo = pr.fields(f)
        ref.append((uo[h, h], vo[h, h], ro[h, h]))
    # FP32 rounding of the stored deviations is absolute, set by the largest velocities of the
    # field (the channels), not by the 1e4-times slower matrix cells: floor 1e-6 of that scale
    umax = max(max(abs(uo), abs(vo)) for uo, vo, _ in ref)
    for (ug, vg, rg), (uo, vo, ro) in zip(vals, ref):
        assert abs(ug - uo) <= 1e-5 * abs(uo) + 1e-6 * umax
        assert abs(vg - vo) <= 1e-5 * abs(vo) + 1e-6 * umax
        assert abs(rg - ro) <= 1e-6
    assert abs(total_drho) / (N * N) < 1e-14


# ------------------------------------------------------------- API behaviour

def test_stop_rule_and_enotconv():
    import torch
    lbm = _lbm()
    kap = np.full((16, 16), 0.05, dtype=np.float32)
    p = lbm.Params(nx=16, ny=16, tau=1.0, eps=1.0, gx=1e-5)
    with lbm.Grid(p, torch.from_numpy(kap).cuda()) as G:
        n, r, ok = G.step(100000, 1e-6, 8)
        assert ok and r <= 1e-6 and n % 8 == 0 and n < 100000
    # a heterogeneous field keeps changing for many steps (a uniform one reaches an exact
    # FP32 fixed point within ~16 steps, where the residual is exactly 0)
    kap2 = synth.lognormal_kappa(16, 16, 3.0, 1.0, seed=8).astype(np.float32)
    with lbm.Grid(p, torch.from_numpy(kap2).cuda()) as G:
        st, n, r = lbm.lbm_step(G.handle, 16, 1e-30, 8)
        assert st == lbm.LBM_ENOTCONV and n == 16 and r > 0


def test_invalid_kappa_detected_on_device():
    import torch
    lbm = _lbm()
    kap = np.full((8, 8), 0.1, dtype=np.float32)
    kap[3, 4] = -1.0
    with pytest.raises(lbm.LbmError) as ei:
        lbm.Grid(lbm.Params(nx=8, ny=8, tau=1.0), torch.from_numpy(kap).cuda())
    assert ei.value.status == lbm.LBM_EINVAL
    kap[3, 4] = np.nan
    with pytest.raises(lbm.LbmError):
        lbm.Grid(lbm.Params(nx=8, ny=8, tau=1.0), torch.from_numpy(kap).cuda())


def test_mean_velocity_bitwise_repeatable_and_checkpoint():
    import torch
    lbm = _lbm()
    kap = synth.lognormal_kappa(64, 64, 6.0, 1.0, seed=9).astype(np.float32)
    p = lbm.Params(nx=64, ny=64, tau=0.8, eps=1.0, gx=1e-6)
    kt = torch.from_numpy(kap).cuda()
    with lbm.Grid(p, kt) as A:
        A.step(100, 0.0, 0)
        m1 = A.mean_velocity()
        assert m1 == A.mean_velocity()
        state = torch.empty(lbm.lbm_grid_state_bytes(A.handle), dtype=torch.uint8, device="cuda")
        t = lbm.lbm_grid_save_state(A.handle, state)
        assert t == 100
        A.step(57, 0.0, 0)
        ref = A.fields()[1].cpu()
        lbm.lbm_grid_load_state(A.handle, state, t)
        A.step(57, 0.0, 0)
        again = A.fields()[1].cpu()
        assert torch.equal(ref, again)
        assert A.steps == 157
    with lbm.Grid(p, kt) as B:
        B.step(100, 0.0, 0)
        assert B.mean_velocity() == m1
    # the header rejects a state saved under other parameters, and the byte count must match
    for other in (lbm.Params(nx=64, ny=64, tau=0.9, eps=1.0, gx=1e-6),
                  lbm.Params(nx=64, ny=64, tau=0.8, eps=1.0, gx=1e-6, storage=2)):
        with lbm.Grid(other, kt) as Cg:
            n_other = lbm.lbm_grid_state_bytes(Cg.handle)
            buf = state if n_other == state.numel() else torch.zeros(n_other, dtype=torch.uint8, device="cuda")
            if buf is not state:
                buf[: state.numel()].copy_(state)
            with pytest.raises(lbm.LbmError) as ei:
                lbm.lbm_grid_load_state(Cg.handle, buf, 100)
            assert ei.value.status == lbm.LBM_EINVAL
    with lbm.Grid(p, kt) as D:
        with pytest.raises(lbm.LbmError) as ei:
            lbm.lbm_grid_load_state(D.handle, state[:-16], 100)
        assert ei.value.status == lbm.LBM_EINVAL
        lbm.lbm_grid_load_state(D.handle, state, t)
        D.step(57, 0.0, 0)
        assert torch.equal(D.fields()[1].cpu(), ref)


@pytest.mark.parametrize("storage,vecs", [(0, (1, 4, 8)), (1, (1, 2, 4, 8)), (2, (1, 2))])
def test_every_cells_per_thread_variant_agrees_bitwise(storage, vecs, monkeypatch):
    """The step is built for several cells-per-thread packs per storage type (the autotuner picks
    one per lattice); each cell's arithmetic is the same in all of them, so the states agree bit for
    bit, with walls and periodic rows alike."""
    import torch
    lbm = _lbm()
    kap = synth.lognormal_kappa(256, 96, 6.0, 1.5, seed=91).astype(np.float32)
    for walls in (False, True):
        states = {}
        for v in vecs:
            monkeypatch.setenv("LBM_STEP_VEC", str(v))
            p = lbm.Params(nx=256, ny=96, tau=0.7, nu=0.05, eps=0.9, gx=2e-6, gy=-1e-6, storage=storage,
                           bc=lbm.LBM_BC_WALLS_Y if walls else lbm.LBM_BC_PERIODIC)
            with lbm.Grid(p, torch.from_numpy(kap).cuda()) as G:
                G.step(150, 0.0, 0)
                st = torch.empty(lbm.lbm_grid_state_bytes(G.handle), dtype=torch.uint8, device="cuda")
                lbm.lbm_grid_save_state(G.handle, st)
                states[v] = st.cpu().numpy()
        for v in vecs[1:]:
            np.testing.assert_array_equal(states[v], states[vecs[0]])
