"""GB300 upscaled lattice Boltzmann library: Python binding of ``liblbm.so``.

The functions named ``lbm_*`` mirror the C ABI of ``include/lbm.h`` one to
one; they only marshal arguments (torch CUDA tensors -> device pointers, the
current torch stream -> ``cuda_stream``). ``Grid`` is a small convenience
wrapper over the same calls. Nothing here computes any part of the method:
every step runs in the library's CUDA kernels, and importing this package
fails when the library is missing.
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

from . import _abi
from ._abi import (LBM_BC_PERIODIC, LBM_BC_WALLS_Y, LBM_ECUDA, LBM_EINVAL, LBM_ENOMEM,  # noqa: F401
                   LBM_ENOTCONV, LBM_ETIMEOUT, LBM_F16, LBM_F32, LBM_F64, LBM_OK)

_abi.lib()   # fail loudly at import when the CUDA library is absent


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_abi.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(status: int, allow=(LBM_OK,)) -> int:
    if status not in allow:
        raise LbmError(status, lbm_last_error())
    return status


def _ptr(t):
    """Device pointer of a CUDA tensor (None -> NULL). Host tensors are passed as
    host pointers on purpose, so the library can reject them with LBM_EINVAL."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        # without a device the library rejects the call before using the stream
        return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


@dataclass
class Params:
    nx: int
    ny: int
    tau: float
    nu: float = -1.0
    eps: float = 1.0
    gx: float = 0.0
    gy: float = 0.0
    bc: int = LBM_BC_PERIODIC
    storage: int = LBM_F32
    scale: float = 0.0
    force_model: int = 0      # 0: simplified Shan-Chen scheme, 1: Guo scheme
    margin: int = 0           # local problems: oversampling margin in cells (0: plain)
    warm_start: int = 0       # local problems: 0 from rest, 1 from the patch's finite-volume Darcy state

    def c(self) -> _abi.lbm_params:
        return _abi.lbm_params(int(self.nx), int(self.ny), float(self.tau), float(self.nu), float(self.eps),
                               float(self.gx), float(self.gy), int(self.bc), int(self.storage), float(self.scale),
                               int(self.force_model), int(self.margin), int(self.warm_start))


# ----------------------------------------------------------------- C ABI mirror

def lbm_last_error() -> str:
    return (_abi.lib().lbm_last_error() or b"").decode()


def lbm_launch_count() -> int:
    return int(_abi.lib().lbm_launch_count())


def lbm_grid_create(params: Params, kappa, g_field=None, stream=None) -> C.c_void_p:
    out = C.c_void_p()
    p = params.c()
    _check(_abi.lib().lbm_grid_create(C.byref(p), _ptr(kappa), _ptr(g_field), _stream(stream), C.byref(out)))
    return out


def lbm_grid_destroy(grid) -> None:
    _check(_abi.lib().lbm_grid_destroy(grid))


def lbm_step(grid, max_steps: int, tol_rel: float = 0.0, check_every: int = 0):
    """Returns (status, steps_done, residual); raises except for LBM_OK / LBM_ENOTCONV."""
    steps = C.c_int64(0)
    res = C.c_double(-1.0)
    st = _check(_abi.lib().lbm_step(grid, int(max_steps), float(tol_rel), int(check_every),
                                    C.byref(steps), C.byref(res)), allow=(LBM_OK, LBM_ENOTCONV))
    return st, int(steps.value), float(res.value)


def lbm_get_fields(grid, rho=None, u=None, v=None) -> None:
    _check(_abi.lib().lbm_get_fields(grid, _ptr(rho), _ptr(u), _ptr(v)))


def lbm_mean_velocity(grid):
    out = (C.c_double * 2)()
    _check(_abi.lib().lbm_mean_velocity(grid, out))
    return float(out[0]), float(out[1])


def lbm_grid_steps(grid) -> int:
    return int(_abi.lib().lbm_grid_steps(grid))


def lbm_grid_state_bytes(grid) -> int:
    return int(_abi.lib().lbm_grid_state_bytes(grid))


CKPT_HEADER_BYTES = 256        # checkpoint header in front of the distribution planes


def _state_bytes(state) -> int:
    """Byte size of a checkpoint tensor; it must be a contiguous CUDA tensor on the current device."""
    import torch
    if not (state.is_cuda and state.is_contiguous()):
        raise ValueError("a checkpoint state must be a contiguous CUDA tensor")
    if state.device.index != torch.cuda.current_device():
        raise ValueError(f"checkpoint state on {state.device}, grid on cuda:{torch.cuda.current_device()}")
    return state.numel() * state.element_size()


def lbm_grid_save_state(grid, state) -> int:
    steps = C.c_int64(0)
    _check(_abi.lib().lbm_grid_save_state(grid, _ptr(state), _state_bytes(state), C.byref(steps)))
    return int(steps.value)


def lbm_grid_load_state(grid, state, steps: int) -> None:
    _check(_abi.lib().lbm_grid_load_state(grid, _ptr(state), _state_bytes(state), int(steps)))


def lbm_grid_scale(grid) -> float:
    return float(_abi.lib().lbm_grid_scale(grid))


def lbm_local_keff_batch(params: Params, kappa, leaves, g_const: float, tol_rel: float, max_steps: int,
                         check_every: int, persistent: bool, keff, status, steps=None, stream=None) -> int:
    """Local problems (Section 3, Eq. 17) for every leaf; ``leaves`` is an int32 CUDA
    tensor [n, 3] of (x0, y0, size). Returns the worst status (OK / ENOTCONV / ETIMEOUT)."""
    n = int(leaves.shape[0])
    p = params.c()
    return _check(_abi.lib().lbm_local_keff_batch(C.byref(p), _ptr(kappa), _ptr(leaves), n, float(g_const),
                                                   float(tol_rel), int(max_steps), int(check_every),
                                                   int(bool(persistent)), _ptr(keff), _ptr(status),
                                                   _ptr(steps), _stream(stream)),
                  allow=(LBM_OK, LBM_ENOTCONV, LBM_ETIMEOUT))


def lbm_set_time_limit(seconds: float) -> None:
    _check(_abi.lib().lbm_set_time_limit(float(seconds)))


def local_keff(params: Params, kappa, leaves, g_const: float = 1e-6, tol_rel: float = 1e-8,
               max_steps: int = 200000, check_every: int = 64, persistent: bool = True, stream=None):
    """Allocating convenience over lbm_local_keff_batch: returns (keff [n,4] f64, status [n], steps [n,2], worst)."""
    import torch
    dev = kappa.device
    n = int(leaves.shape[0])
    keff = torch.empty((n, 4), dtype=torch.float64, device=dev)
    status = torch.empty((n,), dtype=torch.int32, device=dev)
    steps = torch.empty((n, 2), dtype=torch.int32, device=dev)
    worst = lbm_local_keff_batch(params, kappa, leaves, g_const, tol_rel, max_steps, check_every, persistent,
                                 keff, status, steps, stream)
    return keff, status, steps, worst


def local_keff_lg(params: Params, kappa, block: int, coarse, g_const: float = 1e-6, tol_rel: float = 1e-8,
                  max_steps: int = 200000, check_every: int = 64, ring: int = 2, fallback=None, stream=None):
    """Allocating convenience over lbm_local_keff_lg (local-global local problems of every
    block x block block; params.margin >= 2). coarse: float32 [2, 3, ny/block, nx/block] device tensor
    of the coarse runs' (rho - 1, u, v) driven along x, then y; ring 2 = pressure only, 1 = the
    coarse velocity held; fallback: None or float64 [nby, nbx, 4] device tensor of tensors to fall
    back to. Returns (keff [nby, nbx, 4] f64, status [nby, nbx], steps [nby, nbx, 2],
    window [nby, nbx, 2, 4] f64, worst, n_fallback)."""
    import torch
    dev = kappa.device
    nby, nbx = params.ny // block, params.nx // block
    keff = torch.empty((nby, nbx, 4), dtype=torch.float64, device=dev)
    status = torch.empty((nby, nbx), dtype=torch.int32, device=dev)
    steps = torch.empty((nby, nbx, 2), dtype=torch.int32, device=dev)
    window = torch.empty((nby, nbx, 2, 4), dtype=torch.float64, device=dev)
    nfb = C.c_int32(0)
    p = params.c()
    worst = _check(_abi.lib().lbm_local_keff_lg(C.byref(p), _ptr(kappa), int(block), _ptr(coarse), float(g_const),
                                                float(tol_rel), int(max_steps), int(check_every), int(ring),
                                                _ptr(fallback), _ptr(keff), _ptr(status), _ptr(steps), _ptr(window),
                                                C.byref(nfb), _stream(stream)),
                   allow=(LBM_OK, LBM_ENOTCONV, LBM_ETIMEOUT))
    return keff, status, steps, window, worst, int(nfb.value)


def lbm_upscale(params: Params, kappa, block: int, keff_coarse, g_const: float = 1e-6, tol_rel: float = 1e-8,
                max_steps: int = 200000, surrogate=None, spread_max: float = 0.03, stream=None):
    """K* per block x block subdomain (Section 3). Returns (status, n_fallback)."""
    p = params.c()
    nfb = C.c_int32(0)
    sur = getattr(surrogate, "handle", surrogate)
    st = _check(_abi.lib().lbm_upscale(C.byref(p), _ptr(kappa), int(block), sur, float(spread_max),
                                       float(g_const), float(tol_rel), int(max_steps), _ptr(keff_coarse),
                                       C.byref(nfb), _stream(stream)),
                allow=(LBM_OK, LBM_ENOTCONV, LBM_ETIMEOUT))
    return st, int(nfb.value)


def lbm_upscale_lg(params: Params, kappa, block: int, keff_coarse, passes: int = 1, g_const: float = 1e-6,
                   tol_rel: float = 1e-8, max_steps: int = 200000, coarse_max_steps: int = 400000,
                   coarse_tol: float = 1e-7, stream=None):
    """Local-global K* per block x block block in one call (params.margin >= 2; warm_start = 1 for
    the Darcy start). Returns (status, n_fallback of the last pass)."""
    p = params.c()
    nfb = C.c_int32(0)
    st = _check(_abi.lib().lbm_upscale_lg(C.byref(p), _ptr(kappa), int(block), int(passes), float(g_const),
                                          float(tol_rel), int(max_steps), int(coarse_max_steps), float(coarse_tol),
                                          _ptr(keff_coarse), C.byref(nfb), _stream(stream)),
                allow=(LBM_OK, LBM_ENOTCONV, LBM_ETIMEOUT))
    return st, int(nfb.value)


def lbm_coarse_params(params: Params, block: int) -> Params:
    out = _abi.lbm_params()
    p = params.c()
    _check(_abi.lib().lbm_coarse_params(C.byref(p), int(block), C.byref(out)))
    return Params(out.nx, out.ny, out.tau, out.nu, out.eps, out.gx, out.gy, out.bc, out.storage, out.scale,
                  out.force_model, out.margin, out.warm_start)


def lbm_coarse_run(params: Params, block: int, keff_coarse, g_coarse=None, max_steps: int = 100000,
                   tol_rel: float = 0.0, check_every: int = 64, rho=None, u=None, v=None, stream=None):
    """Coarse run with K* (Eq. 18). Returns (status, steps_done)."""
    p = params.c()
    steps = C.c_int64(0)
    st = _check(_abi.lib().lbm_coarse_run(C.byref(p), int(block), _ptr(keff_coarse), _ptr(g_coarse),
                                          int(max_steps), float(tol_rel), int(check_every), _ptr(rho), _ptr(u),
                                          _ptr(v), C.byref(steps), _stream(stream)),
                allow=(LBM_OK, LBM_ENOTCONV))
    return st, int(steps.value)


def lbm_block_average(field, block: int, out=None, stream=None):
    import torch
    ny, nx = field.shape
    if out is None:
        out = torch.empty((ny // block, nx // block), dtype=torch.float32, device=field.device)
    _check(_abi.lib().lbm_block_average(_ptr(field), int(nx), int(ny), int(block), _ptr(out), _stream(stream)))
    return out


SURROGATE_PLANES = 9          # input planes per leaf (lbm_patches)


def lbm_patches(kappa, leaves, x=None, stats=None, stream=None):
    """Surrogate inputs for leaves: x [n, 9, 32, 32] (four phase planes of log K, the size plane, four
    context planes) and stats [n, 3] (CUDA float32)."""
    import torch
    ny, nx = kappa.shape
    n = int(leaves.shape[0])
    if x is None:
        x = torch.empty((n, SURROGATE_PLANES, 32, 32), dtype=torch.float32, device=kappa.device)
    if stats is None:
        stats = torch.empty((n, 3), dtype=torch.float32, device=kappa.device)
    _check(_abi.lib().lbm_patches(_ptr(kappa), int(nx), int(ny), _ptr(leaves), n, _ptr(x), _ptr(stats),
                                  _stream(stream)))
    return x, stats


def lbm_surrogate_param_count() -> int:
    return int(_abi.lib().lbm_surrogate_param_count())


class Surrogate:
    """Owning wrapper of an lbm_surrogate ensemble (the lbm_surrogate_* calls)."""

    def __init__(self, n_models: int = 4, seed: int = 0):
        self.n_models = n_models
        h = C.c_void_p()
        _check(_abi.lib().lbm_surrogate_create(int(n_models), int(seed), C.byref(h)))
        self.handle = h

    def get_params(self, model: int):
        import numpy as np
        out = np.empty(lbm_surrogate_param_count(), dtype=np.float32)
        _check(_abi.lib().lbm_surrogate_get_params(self.handle, int(model), out.ctypes.data))
        return out

    def set_params(self, model: int, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == lbm_surrogate_param_count()
        _check(_abi.lib().lbm_surrogate_set_params(self.handle, int(model), p.ctypes.data))

    def get_normalization(self):
        import numpy as np
        out = np.empty(13, dtype=np.float32)
        _check(_abi.lib().lbm_surrogate_get_normalization(self.handle, out.ctypes.data))
        return out

    def set_normalization(self, norm):
        import numpy as np
        p = np.ascontiguousarray(norm, dtype=np.float32)
        assert p.size == 13
        _check(_abi.lib().lbm_surrogate_set_normalization(self.handle, p.ctypes.data))

    def train(self, x, y, stats, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0, stream=None):
        import numpy as np
        loss = np.zeros((self.n_models, epochs), dtype=np.float32)
        _check(_abi.lib().lbm_surrogate_train(self.handle, _ptr(x), _ptr(y), _ptr(stats), int(x.shape[0]),
                                              int(epochs), int(batch), float(lr), int(seed), loss.ctypes.data,
                                              _stream(stream)))
        return loss

    def predict(self, x, stream=None):
        import torch
        n = int(x.shape[0])
        y = torch.empty((self.n_models, n, 2), dtype=torch.float32, device=x.device)
        _check(_abi.lib().lbm_surrogate_predict(self.handle, _ptr(x), n, _ptr(y), _stream(stream)))
        return y

    def get_gate(self):
        import numpy as np
        out = np.empty(7, dtype=np.float32)
        _check(_abi.lib().lbm_surrogate_get_gate(self.handle, out.ctypes.data))
        return out

    def set_gate(self, spread_by_log2size):
        """Relative spread limits for leaves of 1, 2, 4, ..., 64 cells (used with spread_max = 0)."""
        import numpy as np
        g = np.ascontiguousarray(spread_by_log2size, dtype=np.float32)
        assert g.size == 7
        _check(_abi.lib().lbm_surrogate_set_gate(self.handle, g.ctypes.data))

    def keff(self, params: "Params", kappa, leaves, spread_max: float = 0.0, g_const: float = 1e-6,
             tol_rel: float = 1e-8, max_steps: int = 200000, stream=None):
        """lbm_surrogate_keff: returns (keff [n, 4] f64, fallback [n] i32, status [n] i32, n_fallback, worst)."""
        import torch
        n = int(leaves.shape[0])
        dev = kappa.device
        keff = torch.empty((n, 4), dtype=torch.float64, device=dev)
        fb = torch.empty((n,), dtype=torch.int32, device=dev)
        status = torch.empty((n,), dtype=torch.int32, device=dev)
        nfb = C.c_int32(0)
        p = params.c()
        worst = _check(_abi.lib().lbm_surrogate_keff(self.handle, C.byref(p), _ptr(kappa), _ptr(leaves), n,
                                                     float(spread_max), float(g_const), float(tol_rel),
                                                     int(max_steps), _ptr(keff), _ptr(fb), _ptr(status),
                                                     C.byref(nfb), _stream(stream)),
                       allow=(LBM_OK, LBM_ENOTCONV, LBM_ETIMEOUT))
        return keff, fb, status, int(nfb.value), worst

    def grad(self, model: int, x, t, stream=None):
        """(grad [P], loss, y [n, 2]) of one forward/backward pass (standardised targets t)."""
        import numpy as np
        n = int(x.shape[0])
        g = np.empty(lbm_surrogate_param_count(), dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        y = np.empty((n, 2), dtype=np.float32)
        _check(_abi.lib().lbm_surrogate_grad(self.handle, int(model), _ptr(x), _ptr(t), n, g.ctypes.data,
                                             loss.ctypes.data, y.ctypes.data, _stream(stream)))
        return g, float(loss[0]), y

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _check(_abi.lib().lbm_surrogate_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ convenience

class Grid:
    """Owning wrapper: ``Grid(params, kappa_cuda_f32[, g_field])``."""

    def __init__(self, params: Params, kappa, g_field=None, stream=None):
        self.params = params
        self.stream = stream
        self.handle = lbm_grid_create(params, kappa, g_field, stream)

    def step(self, max_steps: int, tol_rel: float = 0.0, check_every: int = 0):
        st, n, r = lbm_step(self.handle, max_steps, tol_rel, check_every)
        return n, r, st == LBM_OK

    def fields(self):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        shape = (self.params.ny, self.params.nx)
        rho = torch.empty(shape, dtype=torch.float32, device=dev)
        u = torch.empty_like(rho)
        v = torch.empty_like(rho)
        lbm_get_fields(self.handle, rho, u, v)
        return rho, u, v

    def mean_velocity(self):
        return lbm_mean_velocity(self.handle)

    @property
    def steps(self) -> int:
        return lbm_grid_steps(self.handle)

    @property
    def scale(self) -> float:
        return lbm_grid_scale(self.handle)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lbm_grid_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- D3Q19 grids

@dataclass
class Params3D:
    nx: int
    ny: int
    nz: int
    tau: float
    nu: float = -1.0
    eps: float = 1.0
    gx: float = 0.0
    gy: float = 0.0
    gz: float = 0.0
    storage: int = LBM_F32
    margin: int = 0           # oversampling margin of the 3-D local problems

    def c(self) -> _abi.lbm3d_params:
        return _abi.lbm3d_params(int(self.nx), int(self.ny), int(self.nz), float(self.tau), float(self.nu),
                                 float(self.eps), float(self.gx), float(self.gy), float(self.gz), int(self.storage),
                                 int(self.margin))


def lbm3d_grid_create(params: Params3D, kappa, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    p = params.c()
    _check(_abi.lib().lbm3d_grid_create(C.byref(p), _ptr(kappa), _stream(stream), C.byref(h)))
    return h


def lbm3d_coarse_params(params: Params3D, block: int) -> Params3D:
    out = _abi.lbm3d_params()
    p = params.c()
    _check(_abi.lib().lbm3d_coarse_params(C.byref(p), int(block), C.byref(out)))
    return Params3D(nx=out.nx, ny=out.ny, nz=out.nz, tau=out.tau, nu=out.nu, eps=out.eps, gx=out.gx, gy=out.gy,
                    gz=out.gz, storage=out.storage, margin=out.margin)


def lbm3d_coarse_grid_create(fine_params: Params3D, block: int, keff_coarse, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    p = fine_params.c()
    _check(_abi.lib().lbm3d_coarse_grid_create(C.byref(p), int(block), _ptr(keff_coarse), _stream(stream), C.byref(h)))
    return h


def lbm3d_block_average(field, block: int, out=None, stream=None):
    """Mean of a CUDA float32 [nz, ny, nx] field over block^3 cubes -> [nz/b, ny/b, nx/b]."""
    import torch
    nz, ny, nx = (int(v) for v in field.shape)
    if out is None:
        out = torch.empty((nz // block, ny // block, nx // block), dtype=torch.float32, device=field.device)
    _check(_abi.lib().lbm3d_block_average(_ptr(field), nx, ny, nz, int(block), _ptr(out), _stream(stream)))
    return out


def lbm3d_grid_destroy(grid) -> None:
    _check(_abi.lib().lbm3d_grid_destroy(grid))


def lbm3d_step(grid, steps: int) -> None:
    _check(_abi.lib().lbm3d_step(grid, int(steps)))


def lbm3d_get_fields(grid, rho=None, u=None, v=None, w=None) -> None:
    _check(_abi.lib().lbm3d_get_fields(grid, _ptr(rho), _ptr(u), _ptr(v), _ptr(w)))


def lbm3d_mean_velocity(grid):
    out = (C.c_double * 3)()
    _check(_abi.lib().lbm3d_mean_velocity(grid, out))
    return tuple(out)


def lbm3d_local_keff_batch(params: Params3D, kappa, leaves, g_const: float, tol_rel: float, max_steps: int,
                           check_every: int, keff, status, steps=None, stream=None) -> int:
    p = params.c()
    return _check(_abi.lib().lbm3d_local_keff_batch(C.byref(p), _ptr(kappa), _ptr(leaves), int(leaves.shape[0]),
                                                    float(g_const), float(tol_rel), int(max_steps), int(check_every),
                                                    _ptr(keff), _ptr(status), _ptr(steps), _stream(stream)),
                  allow=(LBM_OK, LBM_ENOTCONV, LBM_ETIMEOUT))


def local_keff3(params: Params3D, kappa, leaves, g_const: float = 1e-6, tol_rel: float = 1e-8,
                max_steps: int = 200000, check_every: int = 64, stream=None):
    """Allocating convenience over lbm3d_local_keff_batch: leaves int32 [n, 4] (x0, y0, z0, size);
    returns (keff [n, 3, 3] f64, status [n], steps [n, 3], worst)."""
    import torch
    dev = kappa.device
    n = int(leaves.shape[0])
    keff = torch.empty((n, 3, 3), dtype=torch.float64, device=dev)
    status = torch.empty((n,), dtype=torch.int32, device=dev)
    steps = torch.empty((n, 3), dtype=torch.int32, device=dev)
    worst = lbm3d_local_keff_batch(params, kappa, leaves, g_const, tol_rel, max_steps, check_every, keff, status,
                                   steps, stream)
    return keff, status, steps, worst


def lbm3d_upscale(params: Params3D, kappa, block: int, g_const: float = 1e-6, tol_rel: float = 1e-8,
                  max_steps: int = 200000, keff_coarse=None, stream=None):
    """K* of every block^3 block (3-D local problems, params.margin for oversampling) as a CUDA
    float64 tensor [nz/b, ny/b, nx/b, 3, 3] in fine lattice units; returns (keff, n_notconv, status)."""
    import torch
    if keff_coarse is None:
        keff_coarse = torch.empty((params.nz // block, params.ny // block, params.nx // block, 3, 3),
                                  dtype=torch.float64, device=kappa.device)
    p = params.c()
    nnc = _abi._I32(0)
    st = _check(_abi.lib().lbm3d_upscale(C.byref(p), _ptr(kappa), int(block), float(g_const), float(tol_rel),
                                         int(max_steps), _ptr(keff_coarse), C.byref(nnc), _stream(stream)),
                allow=(LBM_OK, LBM_ENOTCONV, LBM_ETIMEOUT))
    return keff_coarse, int(nnc.value), st


class Grid3D:
    """Owning wrapper of a D3Q19 grid: ``Grid3D(params3d, kappa_cuda_f32 [nz, ny, nx])``, or the
    coarse grid of the upscaled model: ``Grid3D.coarse(fine_params3d, block, keff [nz/b, ny/b, nx/b, 3, 3])``."""

    def __init__(self, params: Params3D, kappa, stream=None, _handle=None):
        self.params = params
        self.handle = _handle if _handle is not None else lbm3d_grid_create(params, kappa, stream)

    @classmethod
    def coarse(cls, fine_params: Params3D, block: int, keff_coarse, stream=None):
        return cls(lbm3d_coarse_params(fine_params, block), None, stream,
                   _handle=lbm3d_coarse_grid_create(fine_params, block, keff_coarse, stream))

    def step(self, steps: int) -> None:
        lbm3d_step(self.handle, steps)

    def fields(self):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        shape = (self.params.nz, self.params.ny, self.params.nx)
        out = [torch.empty(shape, dtype=torch.float32, device=dev) for _ in range(4)]
        lbm3d_get_fields(self.handle, *out)
        return tuple(out)

    def mean_velocity(self):
        return lbm3d_mean_velocity(self.handle)

    def save_state(self, out=None):
        """The grid's state as a CUDA uint8 tensor (or into `out`), for load_state on a grid created
        with the same parameters and field."""
        import torch
        n = int(_abi.lib().lbm3d_grid_state_bytes(self.handle))
        if out is None:
            out = torch.empty((n,), dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
        _check(_abi.lib().lbm3d_grid_save_state(self.handle, _ptr(out), _state_bytes(out)))
        return out

    def load_state(self, state) -> None:
        _check(_abi.lib().lbm3d_grid_load_state(self.handle, _ptr(state), _state_bytes(state)))

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lbm3d_grid_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
