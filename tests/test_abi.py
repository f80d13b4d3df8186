"""The C ABI: the library loads, exports every function include/lbm.h declares,
and rejects invalid arguments on the host (no device work, no GPU needed)."""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    names = set(re.findall(r"\b(lbm(?:3d)?_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1312_0195_gb300 import _abi
    return _abi.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("lbm_grid_create", "lbm_grid_destroy", "lbm_step", "lbm_get_fields",
                     "lbm_mean_velocity", "lbm_last_error", "lbm3d_grid_create", "lbm3d_local_keff_batch",
                     "lbm3d_coarse_grid_create", "lbm3d_block_average", "lbm3d_upscale"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1312_0195_gb300 import _abi
    for name in _declared_functions():
        assert hasattr(lib, name), f"{name} declared in lbm.h but not exported"
        assert name in _abi.SIGNATURES, f"{name} has no Python binding"


def _params(**kw):
    from paper_1312_0195_gb300 import _abi
    base = dict(nx=16, ny=8, tau=1.0, nu=-1.0, eps=1.0, gx=1e-6, gy=0.0, bc=0, storage=0, scale=0.0)
    base.update(kw)
    return _abi.lbm_params(**base)


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-3), dict(tau=0.49), dict(tau=float("nan")),
                                 dict(eps=-0.1), dict(gx=float("inf")), dict(bc=7), dict(storage=3),
                                 dict(scale=3.0), dict(scale=-1.0), dict(nu=float("nan")),
                                 dict(force_model=2)])
def test_create_rejects_bad_params(lib, bad):
    out = C.c_void_p(123)
    p = _params(**bad)
    st = lib.lbm_grid_create(C.byref(p), None, None, None, C.byref(out))
    assert st == 1   # LBM_EINVAL
    assert out.value is None
    assert len(lib.lbm_last_error()) > 0


def test_create_rejects_null_and_host_pointers(lib):
    import numpy as np
    out = C.c_void_p()
    p = _params()
    assert lib.lbm_grid_create(None, None, None, None, C.byref(out)) == 1
    assert lib.lbm_grid_create(C.byref(p), None, None, None, C.byref(out)) == 1
    host = np.ones(16 * 8, dtype=np.float32)
    assert lib.lbm_grid_create(C.byref(p), host.ctypes.data, None, None, C.byref(out)) == 1
    assert b"device pointer" in lib.lbm_last_error()


def test_calls_on_null_grid_are_einval(lib):
    steps = C.c_int64(5)
    res = C.c_double(0.0)
    assert lib.lbm_step(None, 10, 0.0, 0, C.byref(steps), C.byref(res)) == 1
    assert steps.value == 0 and res.value == -1.0
    assert lib.lbm_get_fields(None, None, None, None) == 1
    out = (C.c_double * 2)()
    assert lib.lbm_mean_velocity(None, out) == 1
    assert lib.lbm_grid_destroy(None) == 0
    assert lib.lbm_grid_steps(None) == -1


def test_python_binding_raises_typed_error():
    import paper_1312_0195_gb300 as lbm
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_grid_create(lbm.Params(nx=0, ny=4, tau=1.0), None)
    assert ei.value.status == lbm.LBM_EINVAL


def _params3(**kw):
    from paper_1312_0195_gb300 import _abi
    base = dict(nx=8, ny=8, nz=8, tau=1.0, nu=-1.0, eps=1.0, gx=0.0, gy=0.0, gz=0.0, storage=0, margin=0)
    base.update(kw)
    return _abi.lbm3d_params(**base)


@pytest.mark.parametrize("bad", [dict(nx=0), dict(nz=70000), dict(tau=0.3), dict(eps=-1.0), dict(storage=3),
                                 dict(gz=float("nan"))])
def test_3d_create_rejects_bad_params(lib, bad):
    h = C.c_void_p()
    assert lib.lbm3d_grid_create(C.byref(_params3(**bad)), None, None, C.byref(h)) == 1
    assert not h.value


def test_3d_host_side_validation(lib):
    """The 3-D calls reject invalid sizes, parameters and host pointers before any device work."""
    from paper_1312_0195_gb300 import _abi
    p = _params3()
    out = _abi.lbm3d_params()
    assert lib.lbm3d_coarse_params(C.byref(p), 3, C.byref(out)) == 1           # 8 is not a multiple of 3
    assert lib.lbm3d_coarse_params(C.byref(p), 4, C.byref(out)) == 0
    assert (out.nx, out.ny, out.nz) == (2, 2, 2) and abs(out.tau - 0.625) < 1e-15 and abs(out.nu - 1.0 / 24) < 1e-15
    h = C.c_void_p()
    assert lib.lbm3d_coarse_grid_create(C.byref(p), 4, None, None, C.byref(h)) == 1
    assert lib.lbm3d_block_average(None, 8, 8, 8, 3, None, None) == 1
    host = (C.c_float * 512)()
    assert lib.lbm3d_block_average(host, 8, 8, 8, 4, host, None) == 1              # host pointers
    args = (None, None, 1, 1e-6, 1e-8, 1000, 64, None, None, None, None)
    assert lib.lbm3d_local_keff_batch(C.byref(p), *args) == 1                      # host/NULL pointers
    assert lib.lbm3d_local_keff_batch(C.byref(p), None, None, -1, 1e-6, 1e-8, 1000, 64, None, None, None, None) == 1
    assert lib.lbm3d_local_keff_batch(C.byref(p), None, None, 1, 0.0, 1e-8, 1000, 64, None, None, None, None) == 1
    assert lib.lbm3d_local_keff_batch(C.byref(p), None, None, 1, 1e-6, 1e-8, 0, 64, None, None, None, None) == 1
    assert lib.lbm3d_local_keff_batch(C.byref(p), None, None, 0, 1e-6, 1e-8, 1000, 64, None, None, None, None) == 0
    assert lib.lbm3d_grid_state_bytes(None) == -1
    assert lib.lbm3d_grid_save_state(None, None, 0) == 1 and lib.lbm3d_grid_load_state(None, None, 0) == 1
    nnc = C.c_int32(-1)
    assert lib.lbm3d_upscale(C.byref(p), None, 3, 1e-6, 1e-8, 1000, None, C.byref(nnc), None) == 1   # 8 % 3
    assert nnc.value == 0
    assert lib.lbm3d_upscale(C.byref(p), None, 4, 1e-6, 1e-8, 1000, None, None, None) == 1           # NULL keff


def test_surrogate_keff_rejects_bad_arguments_on_the_host(lib):
    """lbm_surrogate_keff with no ensemble, no params or a negative spread returns LBM_EINVAL
    before any device work."""
    p = _params()
    nfb = C.c_int32(-1)
    assert lib.lbm_surrogate_keff(None, C.byref(p), None, None, 4, 0.03, 1e-6, 0.0, 10, None, None, None,
                                  C.byref(nfb), None) == 1
    assert lib.lbm_surrogate_keff(C.c_void_p(8), None, None, None, 4, 0.03, 1e-6, 0.0, 10, None, None, None,
                                  C.byref(nfb), None) == 1
    assert lib.lbm_surrogate_set_gate(None, None) == 1 and lib.lbm_surrogate_get_gate(None, None) == 1


@pytest.mark.parametrize("bad", [dict(margin=1), dict(margin=0), dict(margin=25), dict(storage=2, margin=15),
                                 dict(warm_start=2), dict(eps=0.0), dict(nx=20), dict(ring=3), dict(check_every=63)])
def test_local_global_rejects_bad_set_ups_on_the_host(lib, bad):
    """lbm_local_keff_lg: margin below 2, block + 2 margin above 64 (45 in FP64), warm_start 2,
    eps = 0 or a field that is not a whole number of blocks give LBM_EINVAL before any device
    work."""
    kw = dict(nx=32, ny=32, margin=4)
    kw.update(bad)
    ring, check_every = kw.pop("ring", 2), kw.pop("check_every", 64)
    p = _params(**kw)
    assert lib.lbm_local_keff_lg(C.byref(p), None, 16, None, 1e-6, 1e-8, 100, check_every, ring, None, None,
                                 None, None, None, None, None) == 1
