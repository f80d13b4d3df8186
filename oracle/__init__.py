"""FP64 CPU oracle of the upscaled LBM -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct restatement of the paper's method (Li & Brown,
Section 2.2 Eqs. 2, 6, 13-16; Section 3 Eqs. 17-18) used to check the CUDA
library. Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline may import it. It shares no code with the CUDA path and the CUDA path
never calls it.

Functions here are thin ctypes marshalling around ``lbm_oracle.c`` plus a few
pure-numpy helpers (dense steady-state solve by brute force, analytic profiles
for the closed-form pins). Parity of every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lbm3d_oracle.c")]
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

Q = 9
# D2Q9 velocities and weights in the paper's order (Section 2): rest, the four axes at angles
# (a - 1) pi / 2, the four diagonals at (a - 5) pi / 2 + pi / 4
EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (-O3, no FMA contraction, OpenMP).

    -O3 without -ffast-math keeps IEEE semantics, and -ffp-contract=off forbids
    fused multiply-adds, so every result is the one the plain C expressions define.
    No -march=native: the same source must build and give the same results on the
    x86 and Arm hosts.

    ``LBM_ORACLE_LIB`` names a prebuilt oracle library to load instead (the
    mutation tests point it at copies with planted mistakes).
    """
    alt = os.environ.get("LBM_ORACLE_LIB")
    if alt:
        return alt
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Thread count of the oracle's OpenMP loops (the CPU baseline is timed at 1 and at all cores)."""
    _L().orc_set_threads(int(n))


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int),
                ("tau", C.c_double), ("nu", C.c_double), ("eps", C.c_double),
                ("walls", C.c_int),
                ("gx", C.c_double), ("gy", C.c_double),
                ("kappa", C.c_void_p), ("ktensor", C.c_void_p), ("gfield", C.c_void_p),
                ("force_model", C.c_int), ("fixed", C.c_void_p)]


_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        _lib.orc_init_rest.argtypes = [C.POINTER(_Problem), dp]
        _lib.orc_velocity.argtypes = [C.POINTER(_Problem), dp, dp, dp, dp]
        _lib.orc_step.argtypes = [C.POINTER(_Problem), dp, dp]
        _lib.orc_run.argtypes = [C.POINTER(_Problem), dp, C.c_void_p, C.c_long, C.c_double, C.c_int,
                                 dp, C.POINTER(C.c_int)]
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_run.restype = C.c_long
        _lib.orc_mean_velocity.argtypes = [C.POINTER(_Problem), dp, dp]
        _lib.orc_local_keff.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_long, C.c_int,
                                        dp, dp, C.POINTER(C.c_long)]
        _lib.orc_local_keff.restype = C.c_int
        _lib.orc_local_keff_os.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_double,
                                           C.c_double, C.c_double, C.c_long, C.c_int,
                                           dp, dp, C.POINTER(C.c_long)]
        _lib.orc_local_keff_os.restype = C.c_int
        _lib.orc_local_keff_from.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_double,
                                             C.c_double, C.c_double, C.c_long, C.c_int, dp,
                                             dp, dp, C.POINTER(C.c_long)]
        _lib.orc_local_keff_from.restype = C.c_int
        _lib.orc_local_lg.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_long, C.c_int, C.c_int, dp, dp, dp, C.POINTER(C.c_long)]
        _lib.orc_local_lg.restype = C.c_int
        _lib.orc_run_mean_steady.argtypes = [C.POINTER(_Problem), dp, C.c_int, C.c_double, C.c_long,
                                             C.c_int, dp, C.POINTER(C.c_int)]
        _lib.orc_run_mean_steady.restype = C.c_long
        _lib.orc_block_average.argtypes = [C.c_int, C.c_int, C.c_int, dp, dp]
        _lib.orc_lattice.argtypes = [C.POINTER(C.c_int), dp]
        _lib.orc3_lattice.argtypes = [C.POINTER(C.c_int), dp]
        _lib.orc3_init_rest.argtypes = [C.POINTER(_Problem3), dp]
        _lib.orc3_step.argtypes = [C.POINTER(_Problem3), dp, dp]
        _lib.orc3_run.argtypes = [C.POINTER(_Problem3), dp, C.c_long]
        _lib.orc3_fields.argtypes = [C.POINTER(_Problem3), dp, dp, dp, dp, dp]
        _lib.orc3_mean_velocity.argtypes = [C.POINTER(_Problem3), dp, dp]
        _lib.orc3_local_keff.argtypes = [C.c_int, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_long, C.c_int, dp, C.POINTER(C.c_long)]
        _lib.orc3_local_keff.restype = C.c_int
        _lib.orc3_local_keff_os.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_double, C.c_double,
                                            C.c_double, C.c_long, C.c_int, dp, C.POINTER(C.c_long)]
        _lib.orc3_local_keff_os.restype = C.c_int
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _Problem3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("tau", C.c_double), ("nu", C.c_double), ("eps", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double), ("gz", C.c_double),
                ("kappa", C.c_void_p), ("ktensor", C.c_void_p)]


Q3 = 19


def lattice3():
    """D3Q19 velocities [19, 3] and weights [19] as the oracle builds them."""
    e = (C.c_int * (Q3 * 3))()
    w = np.empty(Q3)
    _L().orc3_lattice(e, _dp(w))
    return np.array(list(e), dtype=np.int64).reshape(Q3, 3), w


class Problem3D:
    """A periodic D3Q19 problem (Section 2's scheme in three dimensions): ``kappa`` [nz, ny, nx]
    (may contain +inf or 0), or ``ktensor`` [nz, ny, nx, 3, 3] (K*_ij per cell, the coarse run of
    Eq. 18), constant body force ``g`` = (gx, gy, gz)."""

    def __init__(self, tau, nu, eps=1.0, kappa=None, g=(0.0, 0.0, 0.0), ktensor=None):
        if (kappa is None) == (ktensor is None):
            raise ValueError("exactly one of kappa and ktensor is required")
        self.kappa = None if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64)
        self.ktensor = None if ktensor is None else np.ascontiguousarray(ktensor, dtype=np.float64)
        shape = self.kappa.shape if self.kappa is not None else self.ktensor.shape[:3]
        if self.ktensor is not None:
            assert self.ktensor.shape[3:] == (3, 3)
        self.nz, self.ny, self.nx = (int(v) for v in shape)
        self._s = _Problem3(self.nx, self.ny, self.nz, float(tau), float(nu), float(eps),
                            float(g[0]), float(g[1]), float(g[2]),
                            None if self.kappa is None else self.kappa.ctypes.data,
                            None if self.ktensor is None else self.ktensor.ctypes.data)

    def rest(self) -> np.ndarray:
        f = np.empty((self.nz, self.ny, self.nx, Q3))
        _L().orc3_init_rest(C.byref(self._s), _dp(f))
        return f

    def step(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        _L().orc3_step(C.byref(self._s), _dp(f), _dp(out))
        return out

    def run(self, f: np.ndarray, steps: int) -> None:
        assert f.flags.c_contiguous and f.dtype == np.float64
        _L().orc3_run(C.byref(self._s), _dp(f), int(steps))

    def fields(self, f: np.ndarray):
        """(rho, u, v, w) of every cell, each [nz, ny, nx]."""
        out = [np.empty((self.nz, self.ny, self.nx)) for _ in range(4)]
        _L().orc3_fields(C.byref(self._s), _dp(f), *(_dp(o) for o in out))
        return tuple(out)

    def mean_velocity(self, f: np.ndarray) -> np.ndarray:
        m = np.empty(3)
        _L().orc3_mean_velocity(C.byref(self._s), _dp(f), _dp(m))
        return m


def local_keff3(kappa_cube, tau, nu, eps, g_const, tol=1e-8, max_steps=200000, check_every=64, margin=0):
    """Three-dimensional local problem on one periodic s^3 cube (D3Q19), drives along x, y, z;
    Eq. 17 in 3-D. margin > 0: the cube is the leaf grown by `margin` cells on every side
    (oversampling) and the mean velocity is taken over the inner leaf (orc3_local_keff_os).
    Returns dict(keff=[3][3] (K*_ij, i velocity component, j drive), steps=[3], converged=n)."""
    k = np.ascontiguousarray(kappa_cube, dtype=np.float64)
    s = k.shape[0]
    assert k.shape == (s, s, s) and 0 <= margin and s - 2 * margin >= 1
    keff = np.empty(9)
    st = (C.c_long * 3)()
    if margin == 0:
        nconv = _L().orc3_local_keff(s, _dp(k), float(tau), float(nu), float(eps), float(g_const), float(tol),
                                     int(max_steps), int(check_every), _dp(keff), st)
    else:
        nconv = _L().orc3_local_keff_os(s, int(margin), _dp(k), float(tau), float(nu), float(eps), float(g_const),
                                        float(tol), int(max_steps), int(check_every), _dp(keff), st)
    return dict(keff=keff.reshape(3, 3), steps=[st[0], st[1], st[2]], converged=int(nconv))


def grown_cube(field, x0, y0, z0, s, margin):
    """The leaf (x0, y0, z0, s) of a [nz, ny, nx] field grown by `margin` on every side, wrapping
    periodically at the field's edges."""
    nz, ny, nx = field.shape
    zi = (np.arange(z0 - margin, z0 + s + margin) % nz)[:, None, None]
    yi = (np.arange(y0 - margin, y0 + s + margin) % ny)[None, :, None]
    xi = (np.arange(x0 - margin, x0 + s + margin) % nx)[None, None, :]
    return field[zi, yi, xi]


class Problem:
    """One lattice problem: sizes, tau, nu, eps, boundaries, permeability and force.

    ``kappa``: ``[ny, nx]`` scalar permeability (may contain +inf, or 0), or
    ``ktensor``: ``[ny, nx, 4]`` (xx, xy, yx, yy). ``g``: constant (gx, gy) or
    ``gfield``: ``[2, ny, nx]``. ``walls``: half-way bounce-back in y. ``guo``: the
    Guo force scheme of Section 2.1 instead of the simplified scheme of Section 2.2.
    """

    def __init__(self, tau, nu, eps=1.0, kappa=None, ktensor=None, g=(0.0, 0.0), gfield=None,
                 walls=False, guo=False):
        if kappa is None and ktensor is None:
            raise ValueError("kappa or ktensor is required")
        self.kappa = None if kappa is None else np.ascontiguousarray(kappa, dtype=np.float64)
        self.ktensor = None if ktensor is None else np.ascontiguousarray(ktensor, dtype=np.float64)
        shape = (self.kappa if self.kappa is not None else self.ktensor).shape[:2]
        self.ny, self.nx = int(shape[0]), int(shape[1])
        self.gfield = None if gfield is None else np.ascontiguousarray(gfield, dtype=np.float64)
        self._s = _Problem(self.nx, self.ny, float(tau), float(nu), float(eps), int(bool(walls)),
                           float(g[0]), float(g[1]),
                           None if self.kappa is None else self.kappa.ctypes.data,
                           None if self.ktensor is None else self.ktensor.ctypes.data,
                           None if self.gfield is None else self.gfield.ctypes.data,
                           1 if guo else 0)
        self.tau, self.nu, self.eps, self.walls = float(tau), float(nu), float(eps), bool(walls)

    def rest(self) -> np.ndarray:
        f = np.empty((self.ny, self.nx, Q))
        _L().orc_init_rest(C.byref(self._s), _dp(f))
        return f

    def step(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64)
        out = np.empty_like(f)
        _L().orc_step(C.byref(self._s), _dp(f), _dp(out))
        return out

    def run(self, f: np.ndarray, max_steps: int, tol: float = 0.0, check_every: int = 0, work=None):
        """Step ``f`` in place; returns (steps, residual, converged). ``work`` (optional, same shape
        and dtype as f) is the second state the steps alternate with; without it one is allocated
        per call."""
        assert f.flags.c_contiguous and f.dtype == np.float64
        if work is not None:
            assert work.flags.c_contiguous and work.dtype == np.float64 and work.size == f.size
        r = C.c_double(-1.0)
        conv = C.c_int(0)
        n = _L().orc_run(C.byref(self._s), _dp(f), None if work is None else work.ctypes.data, int(max_steps),
                         float(tol), int(check_every), C.byref(r), C.byref(conv))
        return int(n), float(r.value), bool(conv.value)

    def run_mean_steady(self, f: np.ndarray, d: int, tol: float, max_steps: int,
                        check_every: int = 64):
        """Step ``f`` in place until the mean velocity component ``d`` settles.

        Returns (steps, ubar [2], converged); the test is the local-problem one
        of Section 3 (relative change over ``check_every`` steps <= tol * check_every).
        """
        assert f.flags.c_contiguous and f.dtype == np.float64
        ub = np.empty(2)
        conv = C.c_int(0)
        n = _L().orc_run_mean_steady(C.byref(self._s), _dp(f), int(d), float(tol), int(max_steps),
                                     int(check_every), _dp(ub), C.byref(conv))
        return int(n), ub, bool(conv.value)

    def fields(self, f: np.ndarray):
        """(rho, u, v) of the state f, flow velocity of Eq. 15."""
        rho = np.empty((self.ny, self.nx))
        u = np.empty_like(rho)
        v = np.empty_like(rho)
        _L().orc_velocity(C.byref(self._s), _dp(np.ascontiguousarray(f)), _dp(rho), _dp(u), _dp(v))
        return rho, u, v

    def mean_velocity(self, f: np.ndarray) -> np.ndarray:
        out = np.empty(2)
        _L().orc_mean_velocity(C.byref(self._s), _dp(np.ascontiguousarray(f)), _dp(out))
        return out


def lattice():
    e = (C.c_int * 18)()
    w = np.empty(9)
    _L().orc_lattice(e, _dp(w))
    return np.array(list(e), dtype=np.int64).reshape(9, 2), w


def darcy_start(kappa_patch, nu, eps, g_const):
    """The Darcy start of a local problem: for each drive (along x, then y) the distributions
    w_a (rho + 3 e_a . j) of the patch's finite-volume Darcy flow (oracle.surrogate.darcy_solve:
    harmonic face permeabilities, periodic, unit drive), with rho = 1 + 3 eps G p and j = rho u,
    u = (G / nu) times the mean of each cell's two face fluxes along each axis. [2][s][s][9]."""
    from .surrogate import darcy_solve
    k = np.asarray(kappa_patch, dtype=np.float64)
    out = []
    for drive in (0, 1):
        p, qx, qy = darcy_solve(k, drive)
        ux = 0.5 * (qx + np.roll(qx, 1, axis=1)) * g_const / nu
        uy = 0.5 * (qy + np.roll(qy, 1, axis=0)) * g_const / nu
        rho = 1.0 + 3.0 * eps * g_const * p
        jx, jy = rho * ux, rho * uy
        f = np.empty(k.shape + (Q,))
        for a in range(Q):
            f[..., a] = W[a] * (rho + 3.0 * (EX[a] * jx + EY[a] * jy))
        out.append(f)
    return np.ascontiguousarray(np.stack(out))


def local_keff(kappa_leaf, tau, nu, eps, g_const, tol=1e-8, max_steps=200000, check_every=64, margin=0,
               warm=False):
    """Local problems of Section 3 on one periodic square patch; Eq. 17.

    margin > 0: the patch is the leaf with `margin` cells on every side (oversampling, the
    treatment the Conclusions name for channelised media); the stop test and Eq. 17 use the
    mean velocity over the inner leaf only (orc_local_keff_os).
    warm: runs on a patch whose side is a multiple of 8, at least 16, start from the patch's
    Darcy state (darcy_start) instead of rest and stop on the relative change of the whole mean
    velocity vector (orc_local_keff_from); other patches from rest with the plain test.
    Returns dict(keff=[xx, xy, yx, yy], ubar=[u1x, u1y, u2x, u2y], steps=[s1, s2], converged=n).
    """
    k = np.ascontiguousarray(kappa_leaf, dtype=np.float64)
    s = k.shape[0]
    assert k.shape == (s, s) and 0 <= margin and s - 2 * margin >= 1
    keff = np.empty(4)
    ub = np.empty(4)
    st = (C.c_long * 2)()
    if warm and s >= 16 and s % 8 == 0:
        f0 = darcy_start(k, nu, eps, g_const)
        nconv = _L().orc_local_keff_from(s, int(margin), _dp(k), float(tau), float(nu), float(eps), float(g_const),
                                         float(tol), int(max_steps), int(check_every), _dp(f0), _dp(keff), _dp(ub),
                                         st)
    elif margin == 0:
        nconv = _L().orc_local_keff(s, _dp(k), float(tau), float(nu), float(eps), float(g_const),
                                    float(tol), int(max_steps), int(check_every), _dp(keff), _dp(ub), st)
    else:
        nconv = _L().orc_local_keff_os(s, int(margin), _dp(k), float(tau), float(nu), float(eps), float(g_const),
                                       float(tol), int(max_steps), int(check_every), _dp(keff), _dp(ub), st)
    return dict(keff=keff, ubar=ub, steps=[st[0], st[1]], converged=int(nconv))


def coarse_to_fine(fields, r, x0, y0, se):
    """Cell-centred coarse fields [k][ny/r][nx/r] (coarse cell (i, j) covers the fine cells
    [i r, (i + 1) r) x [j r, (j + 1) r)) sampled at the centres of the se x se fine cells from fine
    cell (x0, y0) on (which may lie outside the field: periodic), by bilinear interpolation between
    the four nearest coarse centres, periodic. Returns [k][se][se]."""
    fc = np.asarray(fields, dtype=np.float64)
    _, nyc, nxc = fc.shape
    X = (x0 + np.arange(se) + 0.5) / r - 0.5
    Y = (y0 + np.arange(se) + 0.5) / r - 0.5
    i0 = np.floor(X).astype(np.int64)
    j0 = np.floor(Y).astype(np.int64)
    fx = (X - i0)[None, None, :]
    fy = (Y - j0)[None, :, None]
    i0, i1 = i0 % nxc, (i0 + 1) % nxc
    j0, j1 = j0 % nyc, (j0 + 1) % nyc
    f00 = fc[:, j0][:, :, i0]
    f01 = fc[:, j0][:, :, i1]
    f10 = fc[:, j1][:, :, i0]
    f11 = fc[:, j1][:, :, i1]
    return (1 - fy) * ((1 - fx) * f00 + fx * f01) + fy * ((1 - fx) * f10 + fx * f11)


def local_keff_lg(kappa_ext, margin, state, tau, nu, eps, g_const, tol=1e-8, max_steps=200000, check_every=64,
                  rho_ref=(0.0, 0.0), ring=2):
    """Local-global local problem of one leaf (orc_local_lg): the se x se patch kappa_ext (the leaf
    grown by `margin` >= 1 cells on every side) under the drive G along x, then y, closed by a ring
    of cells fixed at the equilibrium of `state` [2][se][se][3] ((drho, u, v) per cell and drive,
    from a global coarse solution; also the start). K* = nu U F^-1 from the inner window's mean
    velocity U and mean force per unit mass F = G e_d - grad(rho) / (3 eps) (Section 2's Brinkman
    equation at steady state; Eq. 17 when the patch is periodic). rho_ref[d] is subtracted from
    drive d's density deviations first (the library takes the block's own coarse value, so that
    rho0 = 1 sits at the block). ring = 2 (pressure only): the ring keeps the state's density and
    takes its velocity from the inward neighbours at every check (orc_local_lg); ring = 1 keeps the
    state's velocity too.
    Returns dict(keff=[xx, xy, yx, yy], window=[2][4] (mean u, v, d rho/dx, d rho/dy per drive),
    steps=[s1, s2], converged=n)."""
    k = np.ascontiguousarray(kappa_ext, dtype=np.float64)
    se = k.shape[0]
    st0 = np.array(state, dtype=np.float64, order="C")
    assert k.shape == (se, se) and st0.shape == (2, se, se, 3) and margin >= 1 and se - 2 * margin >= 1
    for d in range(2):
        st0[d, ..., 0] -= rho_ref[d]
    win = np.empty(8)
    keff = np.empty(4)
    st = (C.c_long * 2)()
    nconv = _L().orc_local_lg(se, int(margin), _dp(k), float(tau), float(nu), float(eps), float(g_const),
                              float(tol), int(max_steps), int(check_every), int(ring), _dp(st0),
                              _dp(win), _dp(keff), st)
    return dict(keff=keff, window=win.reshape(2, 4), steps=[st[0], st[1]], converged=int(nconv))


def lg_darcy_state(kappa_ext, state, nu, eps, g_const):
    """Start state of a local-global patch from Darcy flow (warm_start = 1 with local-global
    problems): per drive, the finite-volume Darcy flow through the patch (harmonic face
    permeabilities, no wrap) with the ring cells' pressures held at the given state's
    (p = drho / (3 eps G) in unit-drive units, as in darcy_start) and unit drive along the axis;
    interior cells get drho = 3 eps G p and j = rho u with u = (G / nu) times the mean of their two
    face fluxes along each axis; ring cells keep the given state. state, result: [2][se][se][3]."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    k = np.asarray(kappa_ext, dtype=np.float64)
    se = k.shape[0]
    out = np.array(state, dtype=np.float64, order="C")
    ring = np.zeros((se, se), dtype=bool)
    ring[0, :] = ring[-1, :] = ring[:, 0] = ring[:, -1] = True
    inner = np.flatnonzero(~ring.ravel())
    pos = -np.ones(se * se, dtype=np.int64)
    pos[inner] = np.arange(inner.size)
    hx = 2.0 * k[:, :-1] * k[:, 1:] / (k[:, :-1] + k[:, 1:])      # face between (y, x) and (y, x + 1)
    hy = 2.0 * k[:-1, :] * k[1:, :] / (k[:-1, :] + k[1:, :])      # face between (y, x) and (y + 1, x)
    for d in range(2):
        pb = (out[d, ..., 0] / (3.0 * eps * g_const)).ravel()
        rows, cols, vals = [], [], []
        b = np.zeros(inner.size)
        faces = [(y * se + x, y * se + x + 1, hx[y, x], 0) for y in range(se) for x in range(se - 1)] + \
                [(y * se + x, (y + 1) * se + x, hy[y, x], 1) for y in range(se - 1) for x in range(se)]
        for i, j, kf, axis in faces:
            drive = 1.0 if axis == d else 0.0        # e_d . (x_j - x_i)
            for a, c, sgn in ((i, j, 1.0), (j, i, -1.0)):
                if pos[a] < 0:
                    continue
                # flux out of a: kf (p_a - p_c + e_d . (x_c - x_a)); its sum over faces is zero
                rows.append(pos[a]); cols.append(pos[a]); vals.append(kf)
                if pos[c] >= 0:
                    rows.append(pos[a]); cols.append(pos[c]); vals.append(-kf)
                else:
                    b[pos[a]] += kf * pb[c]
                b[pos[a]] -= kf * drive * sgn
        A = sp.csr_matrix((vals, (rows, cols)), shape=(inner.size, inner.size))
        ph = pb.copy()
        ph[inner] = sla.spsolve(A.tocsc(), b)
        P = ph.reshape(se, se)
        qx = hx * (P[:, :-1] - P[:, 1:] + (1.0 if d == 0 else 0.0))   # flux +x through each x-face
        qy = hy * (P[:-1, :] - P[1:, :] + (1.0 if d == 1 else 0.0))
        for y in range(1, se - 1):
            for x in range(1, se - 1):
                drho = 3.0 * eps * g_const * P[y, x]
                rho = 1.0 + drho
                ux = g_const / nu * 0.5 * (qx[y, x - 1] + qx[y, x])
                uy = g_const / nu * 0.5 * (qy[y - 1, x] + qy[y, x])
                out[d, y, x] = (drho, ux, uy)
    return out


def lg_select(keff_lg, window, ok, keff_ref, g_const, eps, cond_max=10.0):
    """Which local-global K* to keep (the library's rule when it is given fallback tensors): a
    block keeps its local-global K*, symmetrised (K*_xy = K*_yx = their mean), when its run met
    the tolerance (ok), that symmetrised tensor is positive definite, and the 2-norm condition
    number of its force matrix F (columns: the two drives' G e_d - grad(rho) / (3 eps)) is at most
    cond_max; otherwise it takes keff_ref. Arrays [n][4], window [n][2][4], ok [n] bool.
    Returns (keff [n][4], used_fallback [n] bool)."""
    k = np.array(keff_lg, dtype=np.float64).reshape(-1, 4)
    w = np.asarray(window, dtype=np.float64).reshape(-1, 2, 4)
    ref = np.asarray(keff_ref, dtype=np.float64).reshape(-1, 4)
    out = np.empty_like(k)
    fb = np.empty(len(k), dtype=bool)
    for i in range(len(k)):
        sym = 0.5 * (k[i, 1] + k[i, 2])
        ks = np.array([[k[i, 0], sym], [sym, k[i, 3]]])
        F = np.array([[g_const - w[i, 0, 2] / (3 * eps), -w[i, 1, 2] / (3 * eps)],
                      [-w[i, 0, 3] / (3 * eps), g_const - w[i, 1, 3] / (3 * eps)]])
        sv = np.linalg.svd(F, compute_uv=False) if np.all(np.isfinite(F)) else np.array([1.0, 0.0])
        good = bool(ok[i]) and np.all(np.isfinite(ks)) and ks[0, 0] > 0 and np.linalg.det(ks) > 0 \
            and sv[1] > 0 and sv[0] / sv[1] <= cond_max
        fb[i] = not good
        out[i] = [ks[0, 0], sym, sym, ks[1, 1]] if good else ref[i]
    return out, fb


def block_average(a, r):
    a = np.ascontiguousarray(a, dtype=np.float64)
    ny, nx = a.shape
    out = np.empty((ny // r, nx // r))
    _L().orc_block_average(nx, ny, r, _dp(a), _dp(out))
    return out


def steady_state_dense(problem: Problem) -> np.ndarray:
    """Brute-force steady state for tiny grids (<= 8x8).

    One oracle step is linear in f (the force enters as rho G and rho is a sum
    of f), so f' = A f. The steady state is the null vector of I - A with the
    mass of the rest state r (mass is conserved, which makes I - A singular).
    Writing f = r + delta: (I - A) delta = A r - r with sum(delta) = 0. A is
    recovered column by column from the step (A e_i = step(r + e_i) - step(r))
    and the system is solved densely with the mass row (least squares, numpy).
    This is a different algorithm from time stepping: it does not iterate.
    """
    n = problem.nx * problem.ny * Q
    if n > 9 * 64:
        raise ValueError("dense steady state is for grids of at most 64 cells")
    r = problem.rest()
    sr = problem.step(r).ravel()
    A = np.empty((n, n))
    for i in range(n):
        e = r.ravel().copy()
        e[i] += 1.0
        A[:, i] = problem.step(e.reshape(r.shape)).ravel() - sr
    M = np.vstack([np.eye(n) - A, np.ones((1, n))])
    rhs = np.concatenate([sr - r.ravel(), [0.0]])
    delta, *_ = np.linalg.lstsq(M, rhs, rcond=None)
    return r + delta.reshape(r.shape)
