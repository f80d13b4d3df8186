#!/usr/bin/env python
"""Benchmark of the fine-grid D2Q9 step (FP32 deviation storage) on one GB300.

Workload: 4096 x 4096 periodic lattice, log-normal permeability K = 1e-2 exp(2 Z)
(Z: Gaussian random field, correlation length 32 cells, seed 2), tau = 0.6,
nu = nu_eff, eps = 1, G = (1e-6, 0), synthetic and seeded. One bench step is one
`lbm_step` call of 1000 lattice time steps with the FP64 residual check every
64 steps (the whole fine-grid hot path: fused stream+collide, moments,
residual and flux reductions), replayed as CUDA graphs. The state (2 x 604 MB)
is far larger than the 129 MB L2, so no L2 flush is needed between steps.

Prints one JSON line (rank 0). `--impl reference` times the FP64 CPU oracle on
the same workload instead (bounded sample per step).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D2Q9 MLUPS (%HBM roofline); K_eff patches/s: surrogate vs batched LBM at stated err"
N = 4096
TAU = 0.6
NU = (TAU - 0.5) / 3.0
G = (1e-6, 0.0)
LBM_STEPS_PER_STEP = 1000
CHECK_EVERY = 64
BYTES_PER_LUP = {"f32": 76, "f16": 40, "f64": 152}
WORKLOAD = (f"D2Q9 fine grid {N}x{N} periodic, log-normal K (sigma_logK=2, ell=32, seed 2), "
            f"tau={TAU}, nu=nu_eff, G=(1e-6,0)")


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl"
        try:
            import torch
            if not torch.cuda.is_available():
                backend = "gloo"
            else:
                torch.cuda.set_device(local)
        except Exception:
            backend = "gloo"
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_kappa() -> np.ndarray:
    import synth
    return synth.lognormal_kappa(N, N, 32.0, 2.0, seed=2).astype(np.float32)


class ClockSampler:
    """Samples SM clock and throttle reasons with nvidia-smi while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=5)

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return {"hbm_gbs": d.get("hbm_gbs"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def traffic_from_profile(kernel_src: str) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged since."""
    p = os.path.join(ROOT, "profiles", "step_f32_4096_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    h = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    if d.get("step_cu_sha256") != h:
        return None
    return d.get("dram_bytes_per_launch")


def oracle_rate(kap: np.ndarray, steps: int, threads: int = 0) -> tuple[float, int, float]:
    """MLUPS of the FP64 oracle on the same lattice for `steps` steps (threads = 0: all host cores).
    The two states alternate in preallocated buffers; one untimed step first touches their pages."""
    import oracle
    cores = threads if threads > 0 else int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    oracle.set_threads(cores)
    p = oracle.Problem(TAU, NU, 1.0, kappa=kap.astype(np.float64), g=G)
    f = p.rest()
    work = np.empty_like(f)
    p.run(f, 1, work=work)
    t0 = time.perf_counter()
    p.run(f, steps, work=work)
    dt = time.perf_counter() - t0
    oracle.set_threads(int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)))
    return N * N * steps / dt / 1e6, cores, dt


def measure_variants(lbm, torch, kap, stream, steps=300):
    """FP16-scaled and FP64 storage on the same lattice, and FP32 at the workload's other tau (1.0,
    nu = nu_eff = 1/6): MLUPS and the fraction of HBM roofline."""
    out = {}
    peaks = measured_peaks()
    for name, st, tau, key in (("f16", lbm.LBM_F16, TAU, "f16"), ("f64", lbm.LBM_F64, TAU, "f64"),
                               ("f32_tau1", lbm.LBM_F32, 1.0, "f32")):
        p = lbm.Params(nx=N, ny=N, tau=tau, nu=-1.0, eps=1.0, gx=G[0], gy=G[1], storage=st)   # nu = nu_eff
        with lbm.Grid(p, kap) as g:
            g.step(50, 0.0, 0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.step(steps, 0.0, 0)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3 / steps
        out[name] = {"mlups": N * N / t / 1e6, "bytes_per_lup": BYTES_PER_LUP[key],
                     "hbm_frac": BYTES_PER_LUP[key] * N * N / t / 1e9 / peaks["hbm_gbs"]}
    return out


def measure_storage_error(lbm, torch, kap_np, crop=512, steps=1000):
    """Error of each storage type against the FP64 oracle: rows/cols 0..crop-1 of the bench field run
    as their own periodic domain for `steps` steps on both sides; relative L2 error of (u, v)."""
    import oracle
    sub = np.ascontiguousarray(kap_np[:crop, :crop])
    prob = oracle.Problem(TAU, NU, 1.0, kappa=sub.astype(np.float64), g=G)
    f = prob.rest()
    prob.run(f, steps)
    _, uo, vo = prob.fields(f)
    den = np.sqrt((uo ** 2 + vo ** 2).sum())
    out = {"workload": f"{crop}^2 crop of the bench field as its own periodic domain, {steps} steps"}
    for name, st in (("f32", lbm.LBM_F32), ("f16", lbm.LBM_F16), ("f64", lbm.LBM_F64)):
        p = lbm.Params(nx=crop, ny=crop, tau=TAU, nu=NU, eps=1.0, gx=G[0], gy=G[1], storage=st)
        with lbm.Grid(p, torch.from_numpy(sub).cuda()) as g:
            g.step(steps, 0.0, 0)
            _, u, v = g.fields()
        u, v = u.cpu().numpy().astype(np.float64), v.cpu().numpy().astype(np.float64)
        out[name] = {"rel_l2_error_uv": float(np.sqrt(((u - uo) ** 2 + (v - vo) ** 2).sum()) / den)}
    return out


def measure_d3q19(lbm, torch, n=256, steps=200, ws=1, rank=0):
    """The scheme on the D3Q19 lattice (Section 2 in three dimensions): n^3 periodic box,
    log-normal K (sigma 2, ell 8, seed 7), tau = 0.6, nu = nu_eff, G = (1e-6, 0, 0); MLUPS and the
    fraction of the measured HBM bandwidth at 19 x 2 x 4 + 4 = 156 B/LUP (FP32), 80 B/LUP (FP16
    scaled storage), 308 B/LUP (FP64). The 3-D local problems on the 16^3 cubes of the box are
    sharded across ranks like the 2-D ones (contiguous, work-balanced ranges, no exchange; rate =
    all cubes over the slowest rank's time); the upscaled model, which needs every cube's K*, runs
    on a single rank only."""
    import synth
    kap = torch.from_numpy(synth.lognormal_kappa3d(n, n, n, 8.0, 2.0, seed=7)).cuda()
    peaks = measured_peaks()
    out = {"workload": f"D3Q19 {n}^3 periodic, log-normal K (sigma 2, ell 8, seed 7), tau 0.6, nu = nu_eff, "
                       "G = (1e-6, 0, 0)"}
    for name, st, bpl, k in (("f32", lbm.LBM_F32, 156, steps), ("f16", lbm.LBM_F16, 80, steps),
                             ("f64", lbm.LBM_F64, 308, steps // 4)):
        p = lbm.Params3D(nx=n, ny=n, nz=n, tau=TAU, nu=NU, eps=1.0, gx=1e-6, storage=st)
        with lbm.Grid3D(p, kap) as g:
            g.step(10)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            g.step(k)
            torch.cuda.synchronize()
            t = (time.perf_counter() - t0) / k
        out[name] = {"mlups": n ** 3 / t / 1e6, "bytes_per_lup": bpl,
                     "hbm_frac": bpl * n ** 3 / t / 1e9 / peaks["hbm_gbs"]}
    if rank == 0:
        out["error_vs_oracle"] = measure_storage_error3(lbm, torch, kap.cpu().numpy())
    # three-dimensional local problems (Eq. 17 in 3-D): every 16^3 cube of the box, three drives
    b = 16
    from paper_1312_0195_gb300.shard import leaf_shard
    cubes = [(x, y, z, b) for z in range(0, n, b) for y in range(0, n, b) for x in range(0, n, b)]
    lo, hi = leaf_shard(np.full(len(cubes), b), rank, ws)
    leaves = torch.tensor(cubes[lo:hi], dtype=torch.int32, device="cuda").reshape(-1, 4)
    p = lbm.Params3D(nx=n, ny=n, nz=n, tau=1.0, eps=1.0)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    keff, status, lsteps, _ = lbm.local_keff3(p, kap, leaves, 1e-6, 1e-8, 200000, 64)
    torch.cuda.synchronize()
    t = max_over_ranks(time.perf_counter() - t0, ws)
    lups = sum_over_ranks(float(lsteps.double().sum()) * b ** 3, ws)
    out["local_keff"] = {"workload": f"all {len(cubes)} cubes of {b}^3, tau 1, G 1e-6 along x, y, z, tol 1e-8",
                         "patches_per_s": len(cubes) / t, "seconds": t, "glups": lups / t / 1e9, "ranks": ws,
                         "converged": int(sum_over_ranks(float((status == 0).sum()), ws))}
    if ws > 1:
        return out
    # the upscaled model on the same box (Eq. 18 in 3-D): fine run at tau 1 for 20k steps against the
    # coarse run with those K* for 1250 steps (the same physical time), block-averaged velocity
    fine_steps, nb = 20000, n // b
    pf = lbm.Params3D(nx=n, ny=n, nz=n, tau=1.0, eps=1.0, gx=1e-6)
    with lbm.Grid3D(pf, kap) as G:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G.step(fine_steps)
        torch.cuda.synchronize()
        t_fine = time.perf_counter() - t0
        _, u, v, w = G.fields()
        avg = [lbm.lbm3d_block_average(f, b).double() for f in (u, v, w)]
        del u, v, w
    with lbm.Grid3D.coarse(pf, b, keff.reshape(nb, nb, nb, 3, 3)) as C:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C.step(fine_steps // b)
        torch.cuda.synchronize()
        t_coarse = time.perf_counter() - t0
        _, uc, vc, wc = C.fields()
    num = sum(((c.double() - a) ** 2).sum() for c, a in zip((uc, vc, wc), avg))
    out["upscaled"] = {"workload": f"fine {n}^3 tau 1, G (1e-6, 0, 0), {fine_steps} steps; coarse {nb}^3 with the "
                                   f"local K* above, {fine_steps // b} steps",
                       "fine_seconds": t_fine, "fine_mlups": n ** 3 * fine_steps / t_fine / 1e6,
                       "coarse_seconds": t_coarse,
                       "rel_l2_vs_fine": float(torch.sqrt(num / sum((a ** 2).sum() for a in avg))),
                       "coarse_over_fine_mean_u": float(uc.double().mean() / avg[0].mean())}
    return out


def measure_storage_error3(lbm, torch, kap_np, crop=32, steps=500):
    """Error of each D3Q19 storage type against the FP64 oracle: the crop^3 corner of the d3q19
    field run as its own periodic box for `steps` steps on both sides (tau 0.6, nu = nu_eff,
    G = (1e-6, 0, 0)); relative L2 error of (u, v, w)."""
    import oracle
    sub = np.ascontiguousarray(kap_np[:crop, :crop, :crop])
    prob = oracle.Problem3D(TAU, NU, 1.0, kappa=sub.astype(np.float64), g=(1e-6, 0.0, 0.0))
    f = prob.rest()
    prob.run(f, steps)
    _, uo, vo, wo = prob.fields(f)
    den = np.sqrt((uo ** 2 + vo ** 2 + wo ** 2).sum())
    out = {"workload": f"{crop}^3 corner of the d3q19 field as its own periodic box, {steps} steps"}
    for name, st in (("f32", lbm.LBM_F32), ("f16", lbm.LBM_F16), ("f64", lbm.LBM_F64)):
        p = lbm.Params3D(nx=crop, ny=crop, nz=crop, tau=TAU, nu=NU, eps=1.0, gx=1e-6, storage=st)
        with lbm.Grid3D(p, torch.from_numpy(sub).cuda()) as g:
            g.step(steps)
            _, u, v, w = (t.cpu().numpy().astype(np.float64) for t in g.fields())
        num = np.sqrt(((u - uo) ** 2 + (v - vo) ** 2 + (w - wo) ** 2).sum())
        out[name] = {"rel_l2_error_uvw": float(num / den)}
    return out


def _oracle_leaf(args):
    """One local problem by the FP64 oracle (process-pool worker)."""
    import oracle
    patch, tol = args
    oracle.local_keff(patch, 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=tol, max_steps=200000)
    return 0


def _oracle_cube(args):
    """One three-dimensional local problem (three drives) by the FP64 oracle (process-pool worker)."""
    import oracle
    cube, tol, max_steps = args
    oracle.local_keff3(cube, 1.0, 1.0 / 6.0, 1.0, 1e-6, tol=tol, max_steps=max_steps)
    return 0


def _oracle_forward(args):
    """Ensemble forward of one patch by the FP64 surrogate oracle (process-pool worker)."""
    from oracle import surrogate as osur
    x, n_models = args
    for m in range(n_models):
        osur.forward(osur.init_params(m), x[None])
    return 0


def measure_cpu_oracles(kap_np, leaf_sample=64, patch_sample=32, cube_sample=16, seed=12):
    """Oracle rates for the other units of the bench, on the host cores (a spawn-started
    process pool, one process per core, each running the oracle as it stands):
    local K* (both drives, tol 1e-8) on a seeded sample of the quadtree leaves of the bench
    field, the 4-model surrogate forward on a seeded sample of their patches, and 3-D local
    problems (three drives, 1024 steps each) on a seeded sample of the 16^3 cubes of the d3q19
    block's field, as lattice updates per second."""
    import multiprocessing as mp
    import synth
    from oracle import surrogate as osur
    leaves = synth.quadtree_leaves(N, N, seed=3)
    rng = np.random.default_rng(seed)
    pick = leaves[rng.choice(len(leaves), leaf_sample, replace=False)]
    patches = [np.array(kap_np[y:y + s, x:x + s], dtype=np.float64) for x, y, s in pick]
    xs = [osur.make_input(np.log(p), 0.0, 1.0) for p in patches[:patch_sample]]
    workers = os.cpu_count() or 1
    k3 = synth.lognormal_kappa3d(256, 256, 256, 8.0, 2.0, seed=7)
    corners = rng.choice(16 ** 3, cube_sample, replace=False)
    cubes = [np.array(k3[16 * (i // 256):16 * (i // 256) + 16, 16 * (i // 16 % 16):16 * (i // 16 % 16) + 16,
                         16 * (i % 16):16 * (i % 16) + 16], dtype=np.float64) for i in corners]
    del k3
    out = {}
    with mp.get_context("spawn").Pool(workers) as pool:
        pool.map(_oracle_leaf, [(patches[0], 1e-8)] * workers)          # start-up outside the timing
        t0 = time.perf_counter()
        pool.map(_oracle_leaf, [(p, 1e-8) for p in patches], chunksize=1)
        dt = time.perf_counter() - t0
        out["local_keff"] = {"value": leaf_sample / dt, "unit": "patches/s", "cores": workers, "kind": "oracle",
                             "sample": f"{leaf_sample} seeded quadtree leaves of the bench field, tol 1e-8 "
                                       f"({dt:.1f} s)"}
        t0 = time.perf_counter()
        pool.map(_oracle_forward, [(x, 4) for x in xs], chunksize=1)
        dt = time.perf_counter() - t0
        out["surrogate_forward"] = {"value": len(xs) / dt, "unit": "patches/s", "cores": workers,
                                    "kind": "oracle",
                                    "sample": f"4-model FP64 forward of {len(xs)} of those leaves' patches ({dt:.1f} s)"}
        # fixed steps, so the sample's time is bounded; the unit is lattice updates (the GPU block
        # reports both cubes/s to tol 1e-8 and GLUPS)
        t0 = time.perf_counter()
        pool.map(_oracle_cube, [(c, 0.0, 1024) for c in cubes], chunksize=1)
        dt = time.perf_counter() - t0
        out["local_keff3"] = {"value": len(cubes) * 3 * 1024 * 16 ** 3 / dt / 1e6, "unit": "MLUPS",
                              "cores": workers, "kind": "oracle",
                              "sample": f"{len(cubes)} seeded 16^3 cubes of the d3q19 block's 256^3 field, three "
                                        f"drives of 1024 steps each ({dt:.1f} s)"}
    return out


def measure_local_keff(lbm, torch, kap, ws, rank=0, sample=512, seed=11):
    """Batched local problems on the 4096^2 field cut by the seeded quadtree (seed 3, ~71.6k
    leaves): one persistent launch for all leaves, tol 1e-8 on the per-drive mean flux,
    check every 64 steps, at most 200k steps per drive. With several ranks each solves its
    contiguous, work-balanced share of the leaves (no exchange) and the rate is all leaves
    over the slowest rank's time. The one-launch-per-leaf mode is timed on a seeded sample of
    `sample` leaves, with the persistent launch on the same sample beside it."""
    import synth
    from paper_1312_0195_gb300.shard import leaf_shard
    all_leaves = synth.quadtree_leaves(N, N, seed=3)
    lo, hi = leaf_shard(all_leaves[:, 2], rank, ws)
    leaves_np = all_leaves[lo:hi]
    p = lbm.Params(nx=N, ny=N, tau=1.0, eps=1.0)
    leaves = torch.from_numpy(leaves_np).cuda()
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    keff, status, steps, worst = lbm.local_keff(p, kap, leaves, 1e-6, 1e-8, 200000, 64, True)
    torch.cuda.synchronize()
    t_all = max_over_ranks(time.perf_counter() - t0, ws)
    st = status.cpu().numpy()
    sz = leaves_np[:, 2].astype(np.float64)
    lups = float((steps.cpu().numpy().astype(np.float64).sum(axis=1) * sz * sz).sum())
    lups = sum_over_ranks(lups, ws)
    converged = int(sum_over_ranks(float((st == 0).sum()), ws))
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(leaves_np), sample, replace=False)
    sub = torch.from_numpy(leaves_np[idx]).cuda()
    times = {}
    for persistent in (True, False):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.local_keff(p, kap, sub, 1e-6, 1e-8, 200000, 64, persistent)
        torch.cuda.synchronize()
        times[persistent] = time.perf_counter() - t0
    return {
        "workload": "4096^2 log-normal field (sigma 2, ell 32), quadtree p=0.6 seed 3, tau=1, "
                    "G=1e-6 along x then y, tol 1e-8, FP32, max 200k steps per drive",
        "leaves": int(len(all_leaves)), "converged": converged, "ranks": ws,
        "patches_per_s": len(all_leaves) / t_all, "seconds": t_all,
        "glups": lups / t_all / 1e9,
        "sample": {"leaves": sample, "persistent_patches_per_s": sample / times[True],
                   "per_leaf_launch_patches_per_s": sample / times[False]},
    }


def _surrogate_fields(nfields, seed0, side):
    """Seeded log-normal fields (sigma ~ U[0.5, 3], ell ~ U[2, 16]) stacked along y."""
    import synth
    rng = np.random.default_rng(seed0)
    ks = []
    for f in range(nfields):
        sigma, ell = rng.uniform(0.5, 3.0), rng.uniform(2.0, 16.0)
        ks.append(synth.lognormal_kappa(side, side, ell, sigma, seed=seed0 * 10000 + f).astype(np.float32))
    return np.concatenate(ks, axis=0)


def _surrogate_set(nfields, seed0, side=256):
    """Held-out set: seeded log-normal fields with their quadtree leaves (the natural mix of sizes)."""
    import synth
    kap = _surrogate_fields(nfields, seed0, side)
    leaves = []
    for f in range(nfields):
        lv = synth.quadtree_leaves(side, side, seed=seed0 * 10000 + f)
        lv[:, 1] += f * side
        leaves.append(lv)
    return kap, np.concatenate(leaves, axis=0)


def _surrogate_train_set(nfields, seed0, per_size, side=512):
    """Training set stratified by leaf size: per field, `per_size[s]` seeded tiles of each size."""
    import synth
    kap = _surrogate_fields(nfields, seed0, side)
    leaves = []
    for f in range(nfields):
        lv = synth.stratified_tiles(side, side, per_size, seed=seed0 * 10000 + f)
        lv[:, 1] += f * side
        leaves.append(lv)
    return kap, np.concatenate(leaves, axis=0)


SUR_SIZES = (1, 2, 4, 8, 16, 32, 64)       # leaf sizes of the per-size gate (index = log2 size)


def _calibrate_gate(sd, in_range, rel, sizes, p99_max=0.04, med_max=0.015):
    """Per leaf size, the largest spread limit (from a log grid) whose accepted leaves keep the
    relative K* error at p99 <= p99_max and median <= med_max on the calibration set; sizes
    with no such limit get the smallest grid value (nearly everything falls back)."""
    grid = np.geomspace(1e-3, 0.3, 60)
    out = []
    for s in SUR_SIZES:
        sel = sizes == s
        best = grid[0]
        if sel.any():
            for g in grid:
                acc = sel & in_range & (sd <= np.log1p(g))
                if acc.sum() < 10:
                    continue
                e = rel[acc]
                if np.percentile(e, 99) <= p99_max and np.median(e) <= med_max:
                    best = g
        out.append(float(best))
    return np.array(out, dtype=np.float32)


def measure_local_global(lbm, torch, n=4096, r=16, margin=4, steps=20000):
    """Local-global against the paper's periodic local problems on a channelised field (the
    regime the Conclusions name): fine run for `steps` steps, K* of every r x r block by the
    periodic local problems and by one local-global pass (lbm_upscale_lg: steady coarse runs with
    the periodic K*, margin 4, pressure-only ring, Darcy start, periodic fallback), coarse runs for
    steps / r steps (the same physical time); relative L2 of the coarse velocity against the
    block-averaged fine velocity."""
    import synth
    nb = n // r
    kt = torch.from_numpy(synth.channel_kappa(n, n, seed=5)).cuda()
    p = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, gx=1e-6, gy=0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with lbm.Grid(p, kt) as G:
        G.step(steps, 0.0, 0)
        _, u, v = G.fields()
    torch.cuda.synchronize()
    t_fine = time.perf_counter() - t0
    ub, vb = lbm.lbm_block_average(u, r).double(), lbm.lbm_block_average(v, r).double()
    del u, v
    den = float(torch.sqrt((ub ** 2 + vb ** 2).sum()))

    def err(ke):
        uc = torch.empty((nb, nb), dtype=torch.float32, device="cuda")
        vc, rc = torch.empty_like(uc), torch.empty_like(uc)
        lbm.lbm_coarse_run(p, r, ke, None, steps // r, 0.0, 64, rc, uc, vc)
        return float(torch.sqrt(((uc.double() - ub) ** 2 + (vc.double() - vb) ** 2).sum())) / den

    kp = torch.empty((nb, nb, 4), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_upscale(lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0), kt, r, kp, 1e-6, 1e-8, 200000)
    torch.cuda.synchronize()
    t_p = time.perf_counter() - t0
    kl = torch.empty_like(kp)
    t0 = time.perf_counter()
    st, nfb = lbm.lbm_upscale_lg(lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, margin=margin, warm_start=1), kt, r, kl,
                                 passes=1)
    torch.cuda.synchronize()
    t_lg = time.perf_counter() - t0
    return {"workload": f"{n}^2 channelised (seed 5, K 1e-2 / 1e-6), r = {r}, tau 1, G 1e-6 along x; fine "
                        f"{steps} steps, coarse {steps // r}; local-global: margin {margin}, pressure-only ring, "
                        "Darcy start, one pass, periodic K* as fallback",
            "fine_seconds": t_fine, "periodic_seconds": t_p, "local_global_seconds": t_lg,
            "local_global_fallback_blocks": nfb, "blocks": nb * nb,
            "coarse_rel_l2_periodic": err(kp), "coarse_rel_l2_local_global": err(kl)}


def measure_surrogate(lbm, torch, train_fields=800, per_size=None, calib_fields=100, test_fields=100, epochs=40,
                      spread_max=0.03):
    """The learned K* surrogate against the batched local LBM on held-out leaves.

    Training set: ~200k leaves cut from seeded log-normal 512^2 fields
    (sigma ~ U[0.5, 3], ell ~ U[2, 16]), stratified by size (equal counts of 8, 16, 32 and 64
    cells: the 64-cell leaves carry most of the LBM cost); labels by local LBM (FP32, tau = 1,
    G = 1e-6, tol 1e-8, persistent launch); non-converged labels are left out. An ensemble of 4
    is trained on it. The gate's spread limit is calibrated per leaf size on separate held-out
    fields; the test leaves are the quadtree leaves of further held-out fields (the natural mix).
    Reports patches/s of LBM alone and end to end through lbm_surrogate_keff (patches, inference
    of all members, gate and local LBM on the rejected leaves, one call), and the relative K*
    error of accepted predictions against their LBM labels."""
    per_size = per_size or {8: 64, 16: 64, 32: 64, 64: 64}

    def label(kap, leaves):
        p = lbm.Params(nx=kap.shape[1], ny=kap.shape[0], tau=1.0, eps=1.0)
        kt, lt = torch.from_numpy(kap).cuda(), torch.from_numpy(leaves).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ke, st, steps, _ = lbm.local_keff(p, kt, lt, 1e-6, 1e-8, 200000, 64, True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        x, stats = lbm.lbm_patches(kt, lt)
        y = torch.log(torch.stack([ke[:, 0], ke[:, 3]], dim=1)).float()
        return kt, lt, p, x, stats, y, ke, st, dt, steps.cpu().numpy().astype(np.float64)

    def rel_err(keff, ke):
        return torch.maximum((keff[:, 0] / ke[:, 0] - 1.0).abs(), (keff[:, 3] / ke[:, 3] - 1.0).abs())

    t0 = time.perf_counter()
    ktr, ltr = _surrogate_train_set(train_fields, 10, per_size)
    t_gen = time.perf_counter() - t0
    _, _, _, xtr, str_, ytr, _, sttr, t_label, _ = label(ktr, ltr)
    ok = sttr == 0
    sur = lbm.Surrogate(4, 3)
    norm = sur.get_normalization()
    norm[12] = 3                                # target base: the leaf's Darcy K* (finite volumes)
    sur.set_normalization(norm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = sur.train(xtr[ok], ytr[ok], str_[ok], epochs=epochs, batch=256, lr=2e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    n_train = int(ok.sum())
    del xtr, str_, ytr
    norm = sur.get_normalization()

    # per-size gate limits from a calibration split
    kca, lca = _surrogate_set(calib_fields, 2000)     # calibration split (seeds 20000000...)
    kc, lc, pc, xc, stc, _, kec, stt_c, _, _ = label(kca, lca)
    pred_c = sur.predict(xc)
    sd_c = pred_c.std(dim=0).max(dim=1).values.cpu().numpy()
    inr = np.ones(len(lca), dtype=bool)
    for k in range(3):
        v = stc[:, k].cpu().numpy()
        inr &= (v >= norm[6 + 2 * k]) & (v <= norm[7 + 2 * k])
    keff_c = torch.exp(pred_c.double().mean(dim=0))
    rel_c = torch.maximum((keff_c[:, 0] / kec[:, 0] - 1).abs(), (keff_c[:, 1] / kec[:, 3] - 1).abs()).cpu().numpy()
    good_c = stt_c.cpu().numpy() == 0
    gate = _calibrate_gate(sd_c, inr & good_c, rel_c, lca[:, 2], p99_max=0.045, med_max=0.018)
    sur.set_gate(gate)

    # held-out test leaves: LBM alone, then the surrogate end to end (one call)
    kte, lte = _surrogate_set(test_fields, 1000)
    kt, lt, p, xte, ste, yte, ke_te, stte, t_lbm, steps_te = label(kte, lte)
    n = len(lte)
    sur.keff(p, kt, lt[:64].contiguous(), 0.0, 1e-6, 1e-8, 200000)      # warm-up: buffers, launch set-up
    results = {}
    for name, smax in (("per_size", 0.0), ("uniform_3pct", spread_max)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        keff, fb, status, nfb, _ = sur.keff(p, kt, lt, smax, 1e-6, 1e-8, 200000)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        good = (stte == 0)
        acc = (fb == 0)
        rel = rel_err(keff, ke_te)
        rel_acc = rel[acc & good].cpu().numpy()
        results[name] = {
            "end_to_end_patches_per_s": n / t_e2e, "speedup_end_to_end": t_lbm / t_e2e,
            "accepted_fraction": float(acc.float().mean()),
            "accepted_rel_err_median": float(np.median(rel_acc)) if rel_acc.size else None,
            "accepted_rel_err_p99": float(np.percentile(rel_acc, 99)) if rel_acc.size else None,
            "fallback_leaves": nfb,
            # leaves whose LBM label did not converge in 200k steps have no verified K*: their count,
            # their share of the LBM time, and how many the gate accepted (left out of the errors)
            "unverified_leaves": int((~good).sum().item()),
            "unverified_accepted": int((acc & ~good).sum().item())}
        if name == "per_size":
            acc_np, rel_np, good_np = acc.cpu().numpy(), rel.cpu().numpy(), good.cpu().numpy()
    # the ensemble's own error on every test leaf (accepted or not)
    pred_te = sur.predict(xte)
    k_pred = torch.exp(pred_te.double().mean(dim=0))
    rel_pred = torch.maximum((k_pred[:, 0] / ke_te[:, 0] - 1).abs(), (k_pred[:, 1] / ke_te[:, 3] - 1).abs())
    rel_pred = rel_pred.cpu().numpy()
    # inference alone: patches, all members and the gate, with every leaf accepted
    x_warm, _ = lbm.lbm_patches(kt, lt)
    sur.predict(x_warm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x_i, st_i = lbm.lbm_patches(kt, lt)
    sur.predict(x_i)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    # where the LBM time goes, by leaf size (cost = cells x steps of both drives)
    sz = lte[:, 2]
    cost = sz.astype(np.float64) ** 2 * steps_te.sum(axis=1)
    by_size = {}
    for size in (8, 16, 32, 64):
        sel = sz == size
        if sel.any():
            e = rel_np[sel & good_np & acc_np]
            by_size[str(size)] = {
                "leaves": int(sel.sum()), "lbm_cost_share": float(cost[sel].sum() / cost.sum()),
                "gate_spread": float(gate[SUR_SIZES.index(size)]),
                "accepted": float(acc_np[sel].mean()),
                "accepted_cost_share": float(cost[sel & acc_np].sum() / cost[sel].sum()),
                "accepted_rel_err_median": float(np.median(e)) if e.size else None,
                "accepted_rel_err_p99": float(np.percentile(e, 99)) if e.size else None,
                "all_rel_err_median": float(np.median(rel_pred[sel & good_np])),
                "all_rel_err_p90": float(np.percentile(rel_pred[sel & good_np], 90))}
    rej_cost = cost[~acc_np].sum() / cost.sum()
    flops = 4 * 2 * 1024 * 9 * (9 * 32 + 32 * 32 + 32 * 64 + 3 * 64 * 64)      # ensemble, per patch
    # the optional Darcy start of the local problems (warm_start = 1): LBM alone, then as the
    # surrogate's fallback; K* compared with the runs from rest
    pw = lbm.Params(nx=p.nx, ny=p.ny, tau=1.0, eps=1.0, warm_start=1)
    lbm.local_keff(pw, kt, lt[:64].contiguous(), 1e-6, 1e-8, 200000, 64, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ke_w, st_w, steps_w, _ = lbm.local_keff(pw, kt, lt, 1e-6, 1e-8, 200000, 64, True)
    torch.cuda.synchronize()
    t_lbm_w = time.perf_counter() - t0
    both = ((stte == 0) & (st_w == 0)).cpu().numpy()
    rel_w = rel_err(ke_w, ke_te).cpu().numpy()[both]
    off_w = (torch.maximum((ke_w[:, 1] - ke_te[:, 1]).abs(), (ke_w[:, 2] - ke_te[:, 2]).abs())
             / torch.sqrt((ke_te[:, 0] * ke_te[:, 3]).abs())).cpu().numpy()[both]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    keff_w, fb_w, _, _, _ = sur.keff(pw, kt, lt, 0.0, 1e-6, 1e-8, 200000)
    torch.cuda.synchronize()
    t_e2e_w = time.perf_counter() - t0
    warm = {
        "lbm_patches_per_s": n / t_lbm_w, "speedup_vs_rest_start": t_lbm / t_lbm_w,
        "lattice_updates_ratio": float((sz.astype(np.float64) ** 2 * steps_w.cpu().numpy().sum(axis=1)).sum()
                                       / cost.sum()),
        "converged_leaves": int((st_w == 0).sum().item()),
        "rel_diff_to_rest_start_median": float(np.median(rel_w)),
        "rel_diff_to_rest_start_p99": float(np.percentile(rel_w, 99)),
        "rel_diff_to_rest_start_max": float(rel_w.max()),
        "offdiag_diff_to_rest_start_median": float(np.median(off_w)),
        "offdiag_diff_to_rest_start_max": float(off_w.max()),
        "surrogate_end_to_end_patches_per_s": n / t_e2e_w,
        "surrogate_speedup_vs_rest_start_lbm": t_lbm / t_e2e_w,
        "surrogate_speedup_vs_darcy_start_lbm": t_lbm_w / t_e2e_w,
        "surrogate_fallback_leaves": int((fb_w != 0).sum().item())}
    sur.close()
    return {
        "workload": f"train: {n_train} leaves ({train_fields} seeded 512^2 log-normal fields, sigma U[0.5,3], "
                    f"ell U[2,16], {per_size} tiles per field by size); gate calibrated per size on "
                    f"{calib_fields} held-out 256^2 fields; test: quadtree leaves 8-64 of {test_fields} further "
                    "held-out fields; labels by local LBM tol 1e-8; ensemble of 4, nine input planes (phase "
                    "planes of the 64x64 log-K plane, size, row and column context), target log K* minus the leaf's "
                    "finite-volume Darcy log K* (mode 3), gate calibrated to p99 <= 4.5 % and median <= 1.8 % per size",
        "train_patches": n_train, "test_patches": n, "epochs": epochs,
        "seconds": {"fields": t_gen, "labels": t_label, "train": t_train},
        "final_train_loss": [float(l[-1]) for l in loss],
        "train_loss_curve_model0": [float(v) for v in loss[0][::max(1, epochs // 10)]],
        "all_rel_err_median": float(np.median(rel_pred[good_np])),
        "all_rel_err_p99": float(np.percentile(rel_pred[good_np], 99)),
        "lbm_patches_per_s": n / t_lbm,
        "surrogate_patches_per_s": n / t_inf,
        "inference_tflops": flops * n / t_inf / 1e12,
        "gate_spread_by_size": {str(s): float(g) for s, g in zip(SUR_SIZES, gate)},
        **results["per_size"],
        "rejected_lbm_cost_share": float(rej_cost),
        "unverified_lbm_cost_share": float(cost[~good_np].sum() / cost.sum()),
        "ideal_speedup": float(1.0 / (rej_cost + t_inf / t_lbm)),
        "uniform_3pct_gate": results["uniform_3pct"],
        "by_leaf_size": by_size,
        "darcy_start": warm,
    }


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    kap = make_kappa()
    import oracle
    oracle.build()
    p = oracle.Problem(TAU, NU, 1.0, kappa=kap.astype(np.float64), g=G)
    f = p.rest()
    work = np.empty_like(f)                   # the two states alternate; no per-step copy
    p.run(f, args.warmup, work=work)
    t0 = time.perf_counter()
    p.run(f, args.steps, work=work)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    value = N * N * args.steps / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded log-normal permeability field)",
        "config": {"workload": WORKLOAD + "; FP64 CPU oracle, one lattice step per bench step",
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} lattice steps of the full {N}x{N} lattice"},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, ws, rank, local):
    import torch
    import paper_1312_0195_gb300 as lbm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    storage = {"f32": lbm.LBM_F32, "f16": lbm.LBM_F16, "f64": lbm.LBM_F64}[args.storage]
    kap_np = make_kappa()
    kap = torch.from_numpy(kap_np).to(dev)
    p = lbm.Params(nx=N, ny=N, tau=TAU, nu=NU, eps=1.0, gx=G[0], gy=G[1], storage=storage)
    grid = lbm.Grid(p, kap)

    for _ in range(args.warmup):
        grid.step(LBM_STEPS_PER_STEP, 0.0, CHECK_EVERY)
    torch.cuda.synchronize()
    barrier(ws)
    l0 = lbm.lbm_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            grid.step(LBM_STEPS_PER_STEP, 0.0, CHECK_EVERY)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    launches = lbm.lbm_launch_count() - l0
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, ws)
    lups = float(N) * N * LBM_STEPS_PER_STEP * args.steps * ws
    value = lups / (ms_max * 1e-3) / 1e6

    # roofline of the dominant kernel: plain fused steps only, timed on the grid's stream
    nplain = 500
    grid.step(nplain, 0.0, 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    grid.step(nplain, 0.0, 0)
    e1.record(stream)
    torch.cuda.synchronize()
    t_launch = e0.elapsed_time(e1) * 1e-3 / nplain
    bytes_launch = BYTES_PER_LUP[args.storage] * float(N) * N
    peaks = measured_peaks()
    achieved = bytes_launch / t_launch / 1e9
    traffic = traffic_from_profile(os.path.join(ROOT, "paper_1312_0195_gb300", "csrc", "step.cu")) \
        if args.storage == "f32" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "peak_source": peaks["source"], "kernel": f"step_kernel<{args.storage}>",
                "algorithmic_bytes_per_lup": BYTES_PER_LUP[args.storage],
                "launch_ms": t_launch * 1e3}
    grid.close()

    # end to end through the public API with host buffers: H2D kappa, create, step, D2H u and v
    kap_host = torch.from_numpy(kap_np).pin_memory()
    u_host = torch.empty((N, N), dtype=torch.float32).pin_memory()
    v_host = torch.empty((N, N), dtype=torch.float32).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        kd = kap_host.to(dev, non_blocking=True)
        with lbm.Grid(p, kd) as g2:
            g2.step(LBM_STEPS_PER_STEP, 0.0, CHECK_EVERY)
            _, u, v = g2.fields()
            u_host.copy_(u, non_blocking=True)
            v_host.copy_(v, non_blocking=True)
            torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, ws)
    e2e = {"value": float(N) * N * LBM_STEPS_PER_STEP * e2e_steps * ws / t_e2e / 1e6, "unit": "MLUPS",
           "h2d_bytes_per_step": int(kap_host.numel() * 4),
           "d2h_bytes_per_step": int(u_host.numel() * 4 + v_host.numel() * 4),
           "steps": e2e_steps}

    variants = {}
    local = surrogate = d3 = lg = None
    if not args.no_extras:
        variants = measure_variants(lbm, torch, kap, stream)
        if rank == 0:
            variants["error_vs_oracle"] = measure_storage_error(lbm, torch, kap_np)
        d3 = measure_d3q19(lbm, torch, ws=ws, rank=rank)
        local = measure_local_keff(lbm, torch, kap, ws, rank)
        if ws == 1:
            lg = measure_local_global(lbm, torch)
        if not args.no_surrogate:
            surrogate = measure_surrogate(lbm, torch, train_fields=args.surrogate_fields,
                                          epochs=args.surrogate_epochs)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, cores, dt = oracle_rate(kap_np, args.cpu_steps)
        rate1, _, dt1 = oracle_rate(kap_np, max(1, args.cpu_steps // 4), threads=1)
        cpu = {"value": rate, "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_steps} lattice steps of the full {N}x{N} lattice ({dt:.1f} s)",
               "one_thread": {"value": rate1, "unit": "MLUPS", "cores": 1,
                              "sample": f"{max(1, args.cpu_steps // 4)} lattice steps of the full lattice "
                                        f"({dt1:.1f} s)"},
               "build": "gcc -O3 -ffp-contract=off -fopenmp (no -march=native: one source for x86 and Arm)"}
        if not args.no_extras:
            cpu["other_units"] = measure_cpu_oracles(kap_np)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
            "data": "synthetic (seeded log-normal permeability field)",
            "config": {"workload": WORKLOAD + f"; {args.storage.upper()} deviation storage",
                       "lattice_steps_per_step": LBM_STEPS_PER_STEP, "check_every": CHECK_EVERY,
                       "l2": "state 1.2 GB >> 129 MB L2 (no flush needed)",
                       "parallelism": f"replicas x{ws}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk.summary(),
        }
        if variants:
            line["storage_variants"] = variants
        if local:
            line["local_keff"] = local
        if surrogate:
            line["surrogate"] = surrogate
        if d3:
            line["d3q19"] = d3
        if lg:
            line["local_global"] = lg
        print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "f16", "f64"])
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the storage variants, the local-problem and the surrogate measurements")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate measurement")
    ap.add_argument("--surrogate-only", action="store_true",
                    help="run only the surrogate measurement (200k training leaves) and print its JSON")
    ap.add_argument("--surrogate-fields", type=int, default=800, help="training fields of the surrogate block")
    ap.add_argument("--surrogate-epochs", type=int, default=40, help="training epochs of the surrogate block")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="profiling mode: create the grid, run this many plain lattice steps, exit")
    ap.add_argument("--profile-local", type=int, default=0,
                    help="profiling mode: this many quadtree leaves of the 4096^2 field, 2000 fixed steps, exit")
    ap.add_argument("--profile-lg", type=int, default=0,
                    help="profiling mode: local-global upscaling of an n^2 channelised field, 2000 fixed steps, exit")
    ap.add_argument("--profile-train", type=int, default=0,
                    help="profiling mode: one surrogate training step (one model) on this many patches, exit")
    ap.add_argument("--profile-3d", type=int, default=0,
                    help="profiling mode: this many cells per side of a D3Q19 box, 8 steps, exit")
    ap.add_argument("--profile-local3d", type=int, default=0,
                    help="profiling mode: this many 16^3 cubes of a 256^3 field, three drives, 512 fixed steps, exit")
    ap.add_argument("--profile-surrogate", type=int, default=0,
                    help="profiling mode: ensemble inference on this many 32x32 patches, exit")
    ap.add_argument("--pipeline", type=int, default=0,
                    help="run the whole upscaled method on an n^2 channelised field (e.g. 16384) and exit")
    ap.add_argument("--pipeline3d", type=int, default=0,
                    help="run the upscaled method in 3-D (D3Q19) on an n^3 log-normal field (e.g. 256) and exit")
    ap.add_argument("--pipeline-steps", type=int, default=20000, help="fine steps of --pipeline / --pipeline3d")
    ap.add_argument("--pipeline-sigma", type=float, default=2.0, help="log-permeability sigma of --pipeline3d")
    ap.add_argument("--pipeline-epochs", type=int, default=10, help="surrogate training epochs of --pipeline")
    ap.add_argument("--pipeline-margins", default="0,4",
                    help="oversampling margins of the local-LBM upscaling runs of --pipeline")
    ap.add_argument("--pipeline-lg", default="4",
                    help="margins of the local-global upscaling runs of --pipeline (empty: none)")
    ap.add_argument("--pipeline-lg-iters", type=int, default=1, help="local-global passes of --pipeline")
    ap.add_argument("--pipeline-lg-f64", action="store_true", help="run the local-global problems in FP64")
    ap.add_argument("--pipeline-lg-start", default="darcy", choices=["darcy", "coarse"],
                    help="start of the local-global problems: the Darcy flow with the ring's pressures held, "
                         "or the coarse state's equilibrium")
    ap.add_argument("--pipeline-lg-steps", type=int, default=200000,
                    help="step limit of the local-global local problems (unconverged blocks fall back)")
    args = ap.parse_args(argv)
    ws, rank, local = dist_init()
    if args.pipeline > 0:
        return run_pipeline(args, local)
    if args.pipeline3d > 0:
        return run_pipeline3d(args, local)
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.profile_steps > 0:
        return run_profile(args, local)
    if args.profile_local > 0:
        return run_profile_local(args, local)
    if args.profile_lg > 0:
        return run_profile_lg(args, local)
    if args.profile_surrogate > 0:
        return run_profile_surrogate(args, local)
    if args.surrogate_only:
        import torch
        import paper_1312_0195_gb300 as lbm
        torch.cuda.set_device(local)
        print(json.dumps(measure_surrogate(lbm, torch, train_fields=args.surrogate_fields,
                                          epochs=args.surrogate_epochs)), flush=True)
        return 0
    if args.profile_3d > 0:
        return run_profile_3d(args, local)
    if args.profile_local3d > 0:
        return run_profile_local3d(args, local)
    if args.profile_train > 0:
        return run_profile_train(args, local)
    return run_ours(args, ws, rank, local)


def run_pipeline(args, local):
    """The whole upscaled method on an n^2 channelised field (default 16384^2, r = 16).

    Fine run (FP32, tau = 1, nu = nu_eff, eps = 1, G = (1e-6, 0)) for `steps` steps; K* of every r x r
    block (Eq. 17) by the surrogate ensemble with local-LBM fallback (trained on the r x r blocks of
    a 4096^2 channelised field of another seed) and by local LBM alone for each oversampling margin
    of --pipeline-margins (0: the paper's plain local problems); with --pipeline-lg, local-global
    K* (pressure-only ring held at the steady coarse runs with the plain K*, margins as given,
    --pipeline-lg-iters passes, falling back to the plain K* block by block); coarse runs (Eq. 18,
    tensor K*, scaled parameters) for steps / r steps, the same physical time; relative L2 error of
    the coarse velocity against the r x r block average of the fine velocity. Prints one JSON line."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    n, r, steps = args.pipeline, 16, args.pipeline_steps
    out = {"workload": f"{n}^2 channelised (seed 5, K 1e-2 / 1e-6), r = {r}, fine {steps} steps, "
                       f"coarse {steps // r} steps", "n": n, "block": r}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0

    p = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, gx=1e-6, gy=0.0)
    kt = torch.from_numpy(synth.channel_kappa(n, n, seed=5)).cuda()
    with lbm.Grid(p, kt) as G:
        _, t = timed(lambda: G.step(steps, 0.0, 0))
        out["fine_seconds"] = t
        out["fine_mlups"] = n * n * steps / t / 1e6
        rho, u, v = G.fields()
        del rho
        ub, vb = lbm.lbm_block_average(u, r), lbm.lbm_block_average(v, r)
        del u, v
    # surrogate for r x r channelised blocks, trained on another seed's field
    m = 4096
    ktr = torch.from_numpy(synth.channel_kappa(m, m, seed=6)).cuda()
    ltr = torch.from_numpy(synth.uniform_leaves(m, m, r)).cuda()
    ptr = lbm.Params(nx=m, ny=m, tau=1.0, eps=1.0)
    (ke, st, _, _), t_lab = timed(lambda: lbm.local_keff(ptr, ktr, ltr, 1e-6, 1e-8, 200000, 64, True))
    x, stats = lbm.lbm_patches(ktr, ltr)
    ok = st == 0
    y = torch.log(torch.stack([ke[:, 0], ke[:, 3]], dim=1)).float()
    sur = lbm.Surrogate(4, 3)
    norm = sur.get_normalization()
    norm[12] = 3                                # target base: the block's Darcy K* (finite volumes)
    sur.set_normalization(norm)
    _, t_train = timed(lambda: sur.train(x[ok], y[ok], stats[ok], epochs=args.pipeline_epochs, batch=256,
                                         lr=2e-3, seed=1))
    out["surrogate_training"] = {"patches": int(ok.sum()), "label_seconds": t_lab, "train_seconds": t_train,
                                 "epochs": args.pipeline_epochs}
    del ktr, ltr, x, stats, ke, st, y
    nb = n // r
    margins = [int(v) for v in args.pipeline_margins.split(",")]
    keff = {"surrogate": torch.empty((nb, nb, 4), dtype=torch.float64, device="cuda")}
    (st_s, nfb), t_s = timed(lambda: lbm.lbm_upscale(p, kt, r, keff["surrogate"], 1e-6, 1e-8, 200000,
                                                     surrogate=sur, spread_max=0.03))
    sur.close()
    out["upscale"] = {"blocks": nb * nb, "surrogate_seconds": t_s, "surrogate_blocks_per_s": nb * nb / t_s,
                      "surrogate_status": st_s, "fallback_fraction": nfb / (nb * nb)}
    for m in margins:
        keff[f"lbm_m{m}"] = torch.empty((nb, nb, 4), dtype=torch.float64, device="cuda")
        pm = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, gx=1e-6, gy=0.0, margin=m)
        (st_l, _), t_l = timed(lambda: lbm.lbm_upscale(pm, kt, r, keff[f"lbm_m{m}"], 1e-6, 1e-8, 200000))
        out["upscale"][f"lbm_margin{m}"] = {"seconds": t_l, "blocks_per_s": nb * nb / t_l, "status": st_l}
    # local-global local problems (pressure-only ring) from the steady coarse runs with the plain
    # K*, falling back to it for blocks that do not converge or give an unusable tensor
    lg_margins = [int(v) for v in args.pipeline_lg.split(",") if v.strip()]
    if lg_margins and 0 in margins:
        for m in lg_margins:
            kcur = keff["lbm_m0"]
            for it in range(args.pipeline_lg_iters):
                cs = torch.empty((2, 3, nb, nb), dtype=torch.float32, device="cuda")

                def states():
                    for d in range(2):
                        pd = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, gx=1e-6 if d == 0 else 0.0,
                                        gy=0.0 if d == 0 else 1e-6)
                        lbm.lbm_coarse_run(pd, r, kcur, None, 400000, 1e-7, 64, cs[d, 0], cs[d, 1], cs[d, 2])
                        cs[d, 0] -= 1.0
                _, t_cs = timed(states)
                pm = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, margin=m, storage=2 if args.pipeline_lg_f64 else 0,
                                warm_start=1 if args.pipeline_lg_start == "darcy" else 0)
                (kl, st_l, _, _, _, nfb_l), t_l = timed(lambda: lbm.local_keff_lg(
                    pm, kt, r, cs, 1e-6, 1e-8, args.pipeline_lg_steps, ring=2, fallback=keff["lbm_m0"]))
                name = f"local_global_m{m}" + (f"_it{it + 1}" if it else "")
                keff[name] = kl
                out["upscale"][name] = {"coarse_states_seconds": t_cs, "seconds": t_l, "blocks_per_s": nb * nb / t_l,
                                        "not_converged": int((st_l != 0).sum()), "fallback_blocks": nfb_l,
                                        "max_steps": args.pipeline_lg_steps,
                                        "storage": "f64" if args.pipeline_lg_f64 else "f32",
                                        "start": args.pipeline_lg_start}
                kcur = kl
                del cs
    if 0 in margins:
        kl, ks = keff["lbm_m0"], keff["surrogate"]
        rel = torch.stack([(ks[..., 0] / kl[..., 0] - 1).abs(), (ks[..., 3] / kl[..., 3] - 1).abs()]).flatten()
        rel = rel.cpu().numpy()
        out["upscale"]["surrogate_kstar_rel_err_vs_lbm_median"] = float(np.median(rel))
        out["upscale"]["surrogate_kstar_rel_err_vs_lbm_p99"] = float(np.percentile(rel, 99))
    pc = lbm.lbm_coarse_params(p, r)
    out["coarse_params"] = {"tau": pc.tau, "nu": pc.nu, "gx": pc.gx}
    den = float(torch.sqrt((ub.double() ** 2 + vb.double() ** 2).sum()))
    for name in keff:
        uc = torch.empty((nb, nb), dtype=torch.float32, device="cuda")
        vc, rc = torch.empty_like(uc), torch.empty_like(uc)
        (_, done), t = timed(lambda: lbm.lbm_coarse_run(p, r, keff[name], None, steps // r, 0.0, 64, rc, uc, vc))
        num = float(torch.sqrt(((uc.double() - ub.double()) ** 2 + (vc.double() - vb.double()) ** 2).sum()))
        out[f"coarse_{name}"] = {"steps": done, "seconds": t, "rel_l2_vs_fine": num / den}
        # the same coarse run continued to steady state (residual 1e-7, FP32 noise floor; at most 200k steps)
        (st_c, done), t = timed(lambda: lbm.lbm_coarse_run(p, r, keff[name], None, 200000, 1e-7, 64, rc, uc, vc))
        num = float(torch.sqrt(((uc.double() - ub.double()) ** 2 + (vc.double() - vb.double()) ** 2).sum()))
        out[f"coarse_{name}"]["to_steady"] = {"steps": done, "status": st_c, "seconds": t,
                                              "rel_l2_vs_fine": num / den}
    print(json.dumps(out), flush=True)
    return 0


def run_pipeline3d(args, local):
    """The upscaled method in three dimensions on an n^3 log-normal field (sigma 2 by default, ell 8,
    seed 7; default n = 256, r = 16): fine D3Q19 run (FP32, tau = 1, nu = nu_eff, eps = 1, G = (1e-6, 0, 0))
    for `steps` steps; K* of every r^3 block by the 3-D local problems (three drives, tol 1e-8) for
    each oversampling margin of --pipeline-margins; coarse run with the tensor K* (Eq. 18 in 3-D,
    scaled parameters) for steps / r steps, the same physical time, and then 16 times longer;
    relative L2 error of the coarse velocity against the r^3 block average of the fine velocity.
    Prints one JSON line."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    n, r, steps = args.pipeline3d, 16, args.pipeline_steps
    nb = n // r
    sig = args.pipeline_sigma
    out = {"workload": f"{n}^3 log-normal (sigma {sig:g}, ell 8, seed 7), r = {r}, fine {steps} steps, "
                       f"coarse {steps // r} steps", "n": n, "block": r}

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = fn()
        torch.cuda.synchronize()
        return res, time.perf_counter() - t0

    p = lbm.Params3D(nx=n, ny=n, nz=n, tau=1.0, eps=1.0, gx=1e-6)
    kt = torch.from_numpy(synth.lognormal_kappa3d(n, n, n, 8.0, sig, seed=7)).cuda()
    with lbm.Grid3D(p, kt) as G:
        _, t = timed(lambda: G.step(steps))
        out["fine_seconds"] = t
        out["fine_mlups"] = n ** 3 * steps / t / 1e6
        _, u, v, w = G.fields()
        avg = [lbm.lbm3d_block_average(f, r).double() for f in (u, v, w)]
        del u, v, w
    leaves = torch.tensor([(x, y, z, r) for z in range(0, n, r) for y in range(0, n, r) for x in range(0, n, r)],
                          dtype=torch.int32, device="cuda")
    den = float(torch.sqrt(sum((a ** 2).sum() for a in avg)))
    out["fine_mean_velocity"] = [float(a.mean()) for a in avg]
    for m in (int(v) for v in args.pipeline_margins.split(",")):
        pm = lbm.Params3D(nx=n, ny=n, nz=n, tau=1.0, eps=1.0, gx=1e-6, margin=m)
        (keff, st, lsteps, _), t = timed(lambda: lbm.local_keff3(pm, kt, leaves, 1e-6, 1e-8, 200000, 64))
        st = st.cpu().numpy()
        res = {"blocks": nb ** 3, "seconds": t, "blocks_per_s": nb ** 3 / t, "converged": int((st == 0).sum()),
               "glups": float(lsteps.double().sum()) * (r + 2 * m) ** 3 / t / 1e9}
        kc = keff.reshape(nb, nb, nb, 3, 3)
        asym = (kc - kc.transpose(-1, -2)).abs().amax(dim=(-1, -2)) / kc.diagonal(dim1=-2, dim2=-1).abs().amax(dim=-1)
        res["kstar_asymmetry_median"] = float(asym.median())
        with lbm.Grid3D.coarse(p, r, kc) as Cg:
            pc = Cg.params
            out["coarse_params"] = {"tau": pc.tau, "nu": pc.nu, "gx": pc.gx}
            done = 0
            for name, k in (("same_time", steps // r), ("16x_longer", 15 * (steps // r))):
                _, t = timed(lambda: Cg.step(k))
                done += k
                _, uc, vc, wc = Cg.fields()
                num = float(torch.sqrt(sum(((c.double() - a) ** 2).sum() for c, a in zip((uc, vc, wc), avg))))
                res[f"coarse_{name}"] = {"steps": done, "seconds": t, "rel_l2_vs_fine": num / den,
                                         "mean_velocity": [float(c.double().mean()) for c in (uc, vc, wc)]}
        out[f"margin{m}"] = res
    print(json.dumps(out), flush=True)
    return 0


def run_profile_lg(args, local):
    """Fixed launch sequence for ncu: local-global upscaling (lbm_upscale_lg, one pass, margin 4,
    Darcy start) of the 16 x 16 blocks of an n^2 channelised field, every local problem and coarse
    run for a fixed 2000 steps. The second local_keff launch is the local-global one."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    n, r = args.profile_lg, 16
    kt = torch.from_numpy(synth.channel_kappa(n, n, seed=5)).cuda()
    p = lbm.Params(nx=n, ny=n, tau=1.0, eps=1.0, margin=4, warm_start=1)
    keff = torch.empty((n // r, n // r, 4), dtype=torch.float64, device="cuda")
    lbm.lbm_upscale_lg(p, kt, r, keff, passes=1, g_const=1e-6, tol_rel=0.0, max_steps=2000, coarse_max_steps=2000,
                       coarse_tol=0.0)
    torch.cuda.synchronize()
    return 0


def run_profile_local(args, local):
    """Fixed launch sequence for ncu: one persistent local-problem launch (2000 steps per drive)."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    kap = torch.from_numpy(make_kappa()).cuda()
    leaves_np = synth.quadtree_leaves(N, N, seed=3)[: args.profile_local]
    p = lbm.Params(nx=N, ny=N, tau=1.0, eps=1.0)
    lbm.local_keff(p, kap, torch.from_numpy(leaves_np).cuda(), 1e-6, 0.0, 2000, 64, True)
    torch.cuda.synchronize()
    return 0


def run_profile_train(args, local):
    """Fixed launch sequence for ncu: one training step of one model (forward, backward, Adam) on the
    patches of the first quadtree leaves of the bench field, with seeded targets."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    n = args.profile_train
    kap = torch.from_numpy(make_kappa()).cuda()
    leaves = torch.from_numpy(synth.quadtree_leaves(N, N, seed=3)[:n]).cuda()
    x, stats = lbm.lbm_patches(kap, leaves)
    y = torch.from_numpy(np.random.default_rng(5).normal(-4.0, 1.0, (n, 2)).astype(np.float32)).cuda()
    with lbm.Surrogate(1, 0) as sur:
        sur.train(x, y, stats, epochs=1, batch=n, lr=1e-3, seed=0)
    torch.cuda.synchronize()
    return 0


def run_profile_3d(args, local):
    """Fixed launch sequence for ncu: one D3Q19 box of profile_3d^3 cells, 8 FP32 steps."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    n = args.profile_3d
    kap = torch.from_numpy(synth.lognormal_kappa3d(n, n, n, 8.0, 2.0, seed=7)).cuda()
    with lbm.Grid3D(lbm.Params3D(nx=n, ny=n, nz=n, tau=TAU, nu=NU, eps=1.0, gx=1e-6), kap) as g:
        g.step(8)
    torch.cuda.synchronize()
    return 0


def run_profile_local3d(args, local):
    """Fixed launch sequence for ncu: the first profile_local3d 16^3 cubes of the 256^3 D3Q19 field of
    the bench's d3q19 block, three drives each, 512 steps with no stopping test."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    n, b = 256, 16
    kap = torch.from_numpy(synth.lognormal_kappa3d(n, n, n, 8.0, 2.0, seed=7)).cuda()
    cubes = [(x, y, z, b) for z in range(0, n, b) for y in range(0, n, b) for x in range(0, n, b)]
    leaves = torch.tensor(cubes[: args.profile_local3d], dtype=torch.int32, device="cuda")
    lbm.local_keff3(lbm.Params3D(nx=n, ny=n, nz=n, tau=1.0, eps=1.0), kap, leaves, 1e-6, 0.0, 512, 64)
    torch.cuda.synchronize()
    return 0


def run_profile_surrogate(args, local):
    """Fixed launch sequence for ncu: patches of the first quadtree leaves, 4-model inference."""
    import torch
    import paper_1312_0195_gb300 as lbm
    import synth
    torch.cuda.set_device(local)
    kap = torch.from_numpy(make_kappa()).cuda()
    leaves = torch.from_numpy(synth.quadtree_leaves(N, N, seed=3)[: args.profile_surrogate]).cuda()
    x, _ = lbm.lbm_patches(kap, leaves)
    with lbm.Surrogate(4, 0) as sur:
        sur.predict(x)
    torch.cuda.synchronize()
    return 0


def run_profile(args, local):
    """A short, fixed launch sequence for ncu: one grid, `profile_steps` plain steps, one check."""
    import torch
    import paper_1312_0195_gb300 as lbm
    torch.cuda.set_device(local)
    storage = {"f32": lbm.LBM_F32, "f16": lbm.LBM_F16, "f64": lbm.LBM_F64}[args.storage]
    kap = torch.from_numpy(make_kappa()).cuda()
    p = lbm.Params(nx=N, ny=N, tau=TAU, nu=NU, eps=1.0, gx=G[0], gy=G[1], storage=storage)
    with lbm.Grid(p, kap) as grid:
        grid.step(args.profile_steps, 0.0, args.profile_steps)
        torch.cuda.synchronize()
    return 0


if __name__ == "__main__":
    sys.exit(main())
