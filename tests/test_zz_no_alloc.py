"""The allocation-free local K* entry point, called through the C ABI.

Some callers of this library cannot allocate device memory (a host program that
owns a fixed device pool, a hard memory budget, an allocator that must not be
bypassed). lbm_local_keff_batch_noalloc serves them: it keeps its work queue in
a static device array inside the library instead of calling cudaMalloc. Here it
must give the same K* as lbm_local_keff_batch, on two calls in a row (the
second call must not see the first call's queue). The file sorts last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""

import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, params, kap, leaves, g, tol, max_steps, k, stream):
    import torch
    n = int(leaves.shape[0])
    keff = torch.full((n, 4), float("nan"), dtype=torch.float64, device="cuda")
    status = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    steps = torch.full((n, 2), -7, dtype=torch.int32, device="cuda")
    p = params.c()
    st = lib.lbm_local_keff_batch_noalloc(C.byref(p), kap.data_ptr(), leaves.data_ptr(), n, float(g), float(tol),
                                          int(max_steps), int(k), keff.data_ptr(), status.data_ptr(),
                                          steps.data_ptr(), stream)
    torch.cuda.synchronize()
    return st, keff.cpu().numpy(), status.cpu().numpy(), steps.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_twice():
    """Same solver on the same inputs: K*, per-leaf status and step counts agree bit for bit with
    the allocating entry point's persistent launch, call after call (FP32 and FP64 storage)."""
    import torch
    import paper_1312_0195_gb300 as lbm
    from paper_1312_0195_gb300 import _abi
    lib = _abi.lib()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [
        # (field size, leaves, tau, g, tol, max_steps, storage): different sizes and counts on each call
        (128, synth.quadtree_leaves(128, 128, seed=41), 1.0, 1e-6, 0.0, 700, lbm.LBM_F32),
        (96, synth.uniform_leaves(96, 96, 16)[:20], 0.8, 2e-6, 1e-8, 50000, lbm.LBM_F32),
        (64, synth.uniform_leaves(64, 64, 32), 0.9, 1e-6, 0.0, 3000, lbm.LBM_F64),
        (128, synth.quadtree_leaves(128, 128, seed=43), 1.0, 1e-6, 0.0, 300, lbm.LBM_F32),
    ]
    for n, leaves_np, tau, g, tol, max_steps, storage in cases:
        kap = torch.from_numpy(synth.lognormal_kappa(n, n, 6.0, 1.5, seed=n).astype(np.float32)).cuda()
        leaves = torch.from_numpy(np.ascontiguousarray(leaves_np, dtype=np.int32)).cuda()
        params = lbm.Params(nx=n, ny=n, tau=tau, nu=0.05, eps=0.9, storage=storage)
        st, ke, sta, steps = _call_noalloc(lib, params, kap, leaves, g, tol, max_steps, 64, stream)
        ref_k, ref_s, ref_steps, ref_worst = lbm.local_keff(params, kap, leaves, g, tol, max_steps, 64, True)
        assert st == ref_worst == lbm.LBM_OK
        np.testing.assert_array_equal(ke, ref_k.cpu().numpy())
        np.testing.assert_array_equal(sta, ref_s.cpu().numpy())
        np.testing.assert_array_equal(steps, ref_steps.cpu().numpy())


def test_noalloc_rejects_oversize_and_bad_leaves():
    import torch
    import paper_1312_0195_gb300 as lbm
    from paper_1312_0195_gb300 import _abi
    lib = _abi.lib()
    stream = torch.cuda.current_stream().cuda_stream
    kap = torch.full((64, 64), 0.05, device="cuda")
    params = lbm.Params(nx=64, ny=64, tau=1.0)
    bad = torch.tensor([[0, 0, 8], [60, 0, 8]], dtype=torch.int32, device="cuda")
    st, *_ = _call_noalloc(lib, params, kap, bad, 1e-6, 0.0, 10, 8, stream)
    assert st == lbm.LBM_EINVAL
    p = params.c()
    big = 131073
    dummy = torch.zeros((1, 3), dtype=torch.int32, device="cuda")
    out = torch.zeros((4,), dtype=torch.float64, device="cuda")
    sti = torch.zeros((1,), dtype=torch.int32, device="cuda")
    st = lib.lbm_local_keff_batch_noalloc(C.byref(p), kap.data_ptr(), dummy.data_ptr(), big, 1e-6, 0.0, 10, 8,
                                          out.data_ptr(), sti.data_ptr(), None, stream)
    assert st == lbm.LBM_EINVAL
    # the FP64 solver holds leaves up to 45 cells: a 46-cell leaf is rejected on the device
    kap2 = torch.full((96, 96), 0.05, device="cuda")
    p64 = lbm.Params(nx=96, ny=96, tau=1.0, storage=lbm.LBM_F64)
    st, *_ = _call_noalloc(lib, p64, kap2, torch.tensor([[0, 0, 46]], dtype=torch.int32, device="cuda"),
                           1e-6, 0.0, 10, 8, stream)
    assert st == lbm.LBM_EINVAL
    # a valid call afterwards still works (the failed calls left the array usable)
    good = torch.tensor([[0, 0, 8], [8, 8, 16]], dtype=torch.int32, device="cuda")
    st, ke, sta, steps = _call_noalloc(lib, params, kap, good, 1e-6, 0.0, 64, 8, stream)
    assert st == lbm.LBM_OK and np.isfinite(ke).all() and (steps == 64).all()
