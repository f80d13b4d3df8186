"""ctypes declarations of include/lbm.h (argument marshalling only).

Loads the in-tree ``liblbm.so``. There is no fallback: if the library is
missing or cannot be loaded, importing the package raises, and every step of
the method runs in the library's CUDA kernels.
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENOTCONV, LBM_ETIMEOUT = range(6)
STATUS_NAMES = {0: "LBM_OK", 1: "LBM_EINVAL", 2: "LBM_ENOMEM", 3: "LBM_ECUDA", 4: "LBM_ENOTCONV",
                5: "LBM_ETIMEOUT"}
LBM_F32, LBM_F16, LBM_F64 = 0, 1, 2
LBM_BC_PERIODIC, LBM_BC_WALLS_Y = 0, 1


class lbm_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32),
                ("tau", C.c_double), ("nu", C.c_double), ("eps", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double),
                ("bc", C.c_int32), ("storage", C.c_int32),
                ("scale", C.c_double), ("force_model", C.c_int32), ("margin", C.c_int32),
                ("warm_start", C.c_int32)]


class lbm3d_params(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("tau", C.c_double), ("nu", C.c_double), ("eps", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double), ("gz", C.c_double),
                ("storage", C.c_int32), ("margin", C.c_int32)]


class lbm3d_leaf(C.Structure):
    _fields_ = [("x0", C.c_int32), ("y0", C.c_int32), ("z0", C.c_int32), ("size", C.c_int32)]


class lbm_leaf(C.Structure):
    _fields_ = [("x0", C.c_int32), ("y0", C.c_int32), ("size", C.c_int32)]


_P = C.c_void_p
_I32 = C.c_int32
_I64 = C.c_int64
_D = C.c_double
_PP = C.POINTER(lbm_params)

# name -> (restype, argtypes); every entry is declared in include/lbm.h
SIGNATURES = {
    "lbm_last_error": (C.c_char_p, []),
    "lbm_launch_count": (_I64, []),
    "lbm_grid_create": (C.c_int, [_PP, _P, _P, _P, C.POINTER(_P)]),
    "lbm_grid_destroy": (C.c_int, [_P]),
    "lbm_step": (C.c_int, [_P, _I64, _D, _I32, C.POINTER(_I64), C.POINTER(_D)]),
    "lbm_get_fields": (C.c_int, [_P, _P, _P, _P]),
    "lbm_mean_velocity": (C.c_int, [_P, C.POINTER(_D)]),
    "lbm_grid_steps": (_I64, [_P]),
    "lbm_grid_state_bytes": (_I64, [_P]),
    "lbm_grid_save_state": (C.c_int, [_P, _P, _I64, C.POINTER(_I64)]),
    "lbm_grid_load_state": (C.c_int, [_P, _P, _I64, _I64]),
    "lbm_grid_scale": (_D, [_P]),
    "lbm_local_keff_batch": (C.c_int, [_PP, _P, _P, _I32, _D, _D, _I64, _I32, _I32, _P, _P, _P, _P]),
    "lbm_set_time_limit": (C.c_int, [_D]),
    "lbm_local_keff_batch_noalloc": (C.c_int, [_PP, _P, _P, _I32, _D, _D, _I64, _I32, _P, _P, _P, _P]),
    "lbm_local_keff_lg": (C.c_int, [_PP, _P, _I32, _P, _D, _D, _I64, _I32, _I32, _P, _P, _P, _P, _P,
                                    C.POINTER(_I32), _P]),
    "lbm_upscale": (C.c_int, [_PP, _P, _I32, _P, _D, _D, _D, _I64, _P, C.POINTER(_I32), _P]),
    "lbm_upscale_lg": (C.c_int, [_PP, _P, _I32, _I32, _D, _D, _I64, _I64, _D, _P, C.POINTER(_I32), _P]),
    "lbm_coarse_params": (C.c_int, [_PP, _I32, _PP]),
    "lbm3d_grid_create": (C.c_int, [C.POINTER(lbm3d_params), _P, _P, C.POINTER(_P)]),
    "lbm3d_grid_destroy": (C.c_int, [_P]),
    "lbm3d_step": (C.c_int, [_P, _I64]),
    "lbm3d_get_fields": (C.c_int, [_P, _P, _P, _P, _P]),
    "lbm3d_mean_velocity": (C.c_int, [_P, C.POINTER(_D)]),
    "lbm3d_local_keff_batch": (C.c_int, [C.POINTER(lbm3d_params), _P, _P, _I32, _D, _D, _I64, _I32, _P, _P, _P, _P]),
    "lbm3d_coarse_params": (C.c_int, [C.POINTER(lbm3d_params), _I32, C.POINTER(lbm3d_params)]),
    "lbm3d_coarse_grid_create": (C.c_int, [C.POINTER(lbm3d_params), _I32, _P, _P, C.POINTER(_P)]),
    "lbm3d_block_average": (C.c_int, [_P, _I32, _I32, _I32, _I32, _P, _P]),
    "lbm3d_upscale": (C.c_int, [C.POINTER(lbm3d_params), _P, _I32, _D, _D, _I64, _P, C.POINTER(_I32), _P]),
    "lbm3d_grid_state_bytes": (_I64, [_P]),
    "lbm3d_grid_save_state": (C.c_int, [_P, _P, _I64]),
    "lbm3d_grid_load_state": (C.c_int, [_P, _P, _I64]),
    "lbm_coarse_run": (C.c_int, [_PP, _I32, _P, _P, _I64, _D, _I32, _P, _P, _P, C.POINTER(_I64), _P]),
    "lbm_block_average": (C.c_int, [_P, _I32, _I32, _I32, _P, _P]),
    "lbm_surrogate_param_count": (_I64, []),
    "lbm_surrogate_create": (C.c_int, [_I32, C.c_uint64, C.POINTER(_P)]),
    "lbm_surrogate_destroy": (C.c_int, [_P]),
    "lbm_surrogate_get_params": (C.c_int, [_P, _I32, _P]),
    "lbm_surrogate_set_params": (C.c_int, [_P, _I32, _P]),
    "lbm_surrogate_set_normalization": (C.c_int, [_P, _P]),
    "lbm_surrogate_get_normalization": (C.c_int, [_P, _P]),
    "lbm_patches": (C.c_int, [_P, _I32, _I32, _P, _I32, _P, _P, _P]),
    "lbm_surrogate_train": (C.c_int, [_P, _P, _P, _P, _I32, _I32, _I32, _D, C.c_uint64, _P, _P]),
    "lbm_surrogate_predict": (C.c_int, [_P, _P, _I32, _P, _P]),
    "lbm_surrogate_grad": (C.c_int, [_P, _I32, _P, _P, _I32, _P, _P, _P, _P]),
    "lbm_surrogate_set_gate": (C.c_int, [_P, _P]),
    "lbm_surrogate_get_gate": (C.c_int, [_P, _P]),
    "lbm_surrogate_keff": (C.c_int, [_P, _P, _P, _P, _I32, _D, _D, _D, _I64, _P, _P, _P, C.POINTER(_I32), _P]),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded liblbm.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; g.build()\"` "
                "(needs nvcc); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return sorted(SIGNATURES)
