"""Permeability and body-force fields, seeded.

Every array is indexed ``[y, x]`` (row = y, x fastest) with cell-centred
coordinates ``x_i = (i + 1/2) dx`` for 0-based ``i``. The paper's analytic
fields are Eq. 22 (Section 4.1), the layers and checkerboard of Section 4.2,
Eq. 23 and Eq. 24 (Section 4.3.1). The random fields stand in for the
log-normal and channelised media the method is meant for.
"""

from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian_random_field(nx: int, ny: int, ell: float, seed: int,
                          covariance: str = "exp_r2_over_2l2") -> np.ndarray:
    """Stationary periodic Gaussian field Z with sample mean 0 and variance 1.

    Spectral synthesis: white noise from PCG64(seed) is filtered in Fourier
    space by the square root of the spectral density of the covariance
    ``C(r) = exp(-r^2 / (2 ell^2))`` (default) or ``exp(-r^2 / ell^2)``, then
    standardised with its own sample mean and standard deviation.
    """
    rng = _rng(seed)
    white = rng.standard_normal((ny, nx))
    kx = 2.0 * np.pi * np.fft.fftfreq(nx)
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    if covariance == "exp_r2_over_2l2":
        spec = np.exp(-0.5 * ell * ell * k2)
    elif covariance == "exp_r2_over_l2":
        spec = np.exp(-0.25 * ell * ell * k2)
    else:
        raise ValueError(f"unknown covariance {covariance!r}")
    z = np.fft.ifft2(np.fft.fft2(white) * np.sqrt(spec)).real
    z -= z.mean()
    sd = z.std()
    if sd == 0.0:
        raise ValueError("degenerate random field (zero variance)")
    return z / sd


def lognormal_kappa(nx: int, ny: int, ell: float, sigma: float, seed: int,
                    k0: float = 1e-2) -> np.ndarray:
    """Log-normal permeability ``K = k0 * exp(sigma * Z)`` (float64)."""
    return k0 * np.exp(sigma * gaussian_random_field(nx, ny, ell, seed))


def lognormal_kappa3d(nx: int, ny: int, nz: int, ell: float, sigma: float, seed: int,
                      k0: float = 1e-2) -> np.ndarray:
    """Three-dimensional log-normal permeability ``[nz, ny, nx]`` (float32): the recipe of
    ``gaussian_random_field`` (white noise from PCG64(seed), spectral filter of
    ``exp(-r^2 / (2 ell^2))``, standardised) on a periodic box, then ``k0 exp(sigma Z)``."""
    rng = _rng(seed)
    white = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    k2 = (2.0 * np.pi * np.fft.fftfreq(nz))[:, None, None] ** 2 + \
        (2.0 * np.pi * np.fft.fftfreq(ny))[None, :, None] ** 2 + \
        (2.0 * np.pi * np.fft.rfftfreq(nx))[None, None, :] ** 2
    z = np.fft.irfftn(np.fft.rfftn(white) * np.sqrt(np.exp(-0.5 * ell * ell * k2)), s=(nz, ny, nx),
                      axes=(0, 1, 2))
    z -= z.mean()
    sd = z.std()
    if sd == 0.0:
        raise ValueError("degenerate random field (zero variance)")
    return (k0 * np.exp(sigma * z / sd)).astype(np.float32)


def quadtree_leaves(nx: int, ny: int, seed: int, root: int = 64, min_size: int = 8,
                    p_split: float = 0.6) -> np.ndarray:
    """Seeded quadtree over ``root``-sized tiles; returns int32 ``[n, 3]`` of (x0, y0, size).

    A node larger than ``min_size`` splits into four children with probability
    ``p_split``; the expected number of leaves per 64-cell root at p = 0.6 is 17.49.
    Leaves are emitted root by root in row-major order, depth first.
    """
    if nx % root or ny % root:
        raise ValueError("field size must be a multiple of the root size")
    rng = _rng(seed)
    out = []
    for ry in range(0, ny, root):
        for rx in range(0, nx, root):
            stack = [(rx, ry, root)]
            while stack:
                x, y, s = stack.pop()
                if s > min_size and rng.random() < p_split:
                    h = s // 2
                    stack.extend([(x + h, y + h, h), (x, y + h, h), (x + h, y, h), (x, y, h)])
                else:
                    out.append((x, y, s))
    return np.asarray(out, dtype=np.int32).reshape(-1, 3)


def stratified_tiles(nx: int, ny: int, per_size: dict, seed: int) -> np.ndarray:
    """Seeded leaf set with a fixed count per size: for each size s, ``per_size[s]`` distinct
    s-aligned tiles of the field (all of them when the field has fewer). int32 ``[n, 3]``."""
    rng = _rng(seed)
    out = []
    for size in sorted(per_size):
        tiles = uniform_leaves(nx, ny, size)
        k = min(int(per_size[size]), len(tiles))
        out.append(tiles[np.sort(rng.choice(len(tiles), k, replace=False))])
    return np.concatenate(out, axis=0).astype(np.int32)


def uniform_leaves(nx: int, ny: int, size: int) -> np.ndarray:
    """Row-major tiling of the field into ``size``-square blocks, int32 ``[n, 3]``."""
    if nx % size or ny % size:
        raise ValueError("field size must be a multiple of the block size")
    ys, xs = np.meshgrid(np.arange(0, ny, size), np.arange(0, nx, size), indexing="ij")
    n = xs.size
    return np.stack([xs.ravel(), ys.ravel(), np.full(n, size)], axis=1).astype(np.int32)


def channel_kappa(nx: int, ny: int, seed: int, k_high: float = 1e-2, k_low: float = 1e-6,
                  spacing: int = 128, width=(4, 12)) -> np.ndarray:
    """Sinuous high-permeability channels over a low-permeability matrix (float32).

    ``ny // spacing`` channels; channel c has centre line
    ``y = y0 + A sin(2 pi x / lam + phi)`` (periodic in y), an integer width
    drawn from ``width`` (inclusive), wavelength ``lam ~ U[nx/32, nx/4]`` and
    amplitude ``A ~ U[4, lam / (4 pi)]`` so the centre line's slope stays <= 1/2.
    """
    rng = _rng(seed)
    kap = np.full((ny, nx), k_low, dtype=np.float32)
    xs = np.arange(nx, dtype=np.float64) + 0.5
    cols = np.arange(nx)
    nch = max(1, ny // spacing)
    for _ in range(nch):
        y0 = rng.uniform(0, ny)
        lam = rng.uniform(max(16.0, nx / 32.0), max(32.0, nx / 4.0))
        amp = rng.uniform(4.0, max(4.0, lam / (4.0 * np.pi)))
        phi = rng.uniform(0, 2 * np.pi)
        w = int(rng.integers(width[0], width[1] + 1))
        yc = y0 + amp * np.sin(2 * np.pi * xs / lam + phi)
        base = np.floor(yc - w / 2.0 + 0.5).astype(np.int64)
        for dy in range(w):
            kap[(base + dy) % ny, cols] = k_high
    return kap


def block_kappa_eq22(n: int = 100, k_in: float = 1e-6, k_out: float = 1e-5) -> np.ndarray:
    """Eq. 22: ``k_in`` at 1-based indices 31 <= i, j <= 70 of a 100x100 grid, else ``k_out``."""
    kap = np.full((n, n), k_out)
    lo, hi = (30 * n) // 100, (70 * n) // 100
    kap[lo:hi, lo:hi] = k_in
    return kap


def layered_kappa(nx: int, ny: int, k1: float, k2: float, n_layers: int = 10) -> np.ndarray:
    """Section 4.2.1: ``n_layers`` equal layers parallel to y (kappa varies along x).

    The 1st, 3rd, ... layers (1-based) hold ``k1``; the even layers hold ``k2``.
    """
    if nx % n_layers:
        raise ValueError("nx must be a multiple of the layer count")
    w = nx // n_layers
    layer = np.arange(nx) // w
    row = np.where(layer % 2 == 0, k1, k2)
    return np.broadcast_to(row[None, :], (ny, nx)).copy()


def checkerboard_kappa(n: int, k1: float, k2: float, n_squares: int = 10) -> np.ndarray:
    """Section 4.2.2: ``n_squares`` x ``n_squares`` squares alternating ``k1`` / ``k2``."""
    if n % n_squares:
        raise ValueError("n must be a multiple of the square count")
    w = n // n_squares
    idx = np.arange(n) // w
    par = (idx[:, None] + idx[None, :]) % 2
    return np.where(par == 0, k1, k2).astype(np.float64)


def _fiveblock_mask(xc: np.ndarray, yc: np.ndarray) -> np.ndarray:
    def box(x0, x1, y0, y1):
        return (xc >= x0) & (xc <= x1) & (yc >= y0) & (yc <= y1)
    return (box(0.45, 0.55, 0.45, 0.55) | box(0.2, 0.3, 0.2, 0.3) | box(0.7, 0.8, 0.7, 0.8)
            | box(0.2, 0.3, 0.7, 0.8) | box(0.7, 0.8, 0.2, 0.3))


def fiveblock_kappa_eq23(n: int = 400, k_const: float = 1.0, length: float = 1.0) -> np.ndarray:
    """Eq. 23 on an ``n`` x ``n`` cell-centred grid of a ``length``-sided square.

    ``k_const`` inside the five square blocks, ``10 (1 + sin(80 pi x) cos(80 pi y)) k_const``
    elsewhere (x, y in metres).
    """
    dx = length / n
    c = (np.arange(n) + 0.5) * dx
    yc, xc = np.meshgrid(c, c, indexing="ij")
    sinus = 10.0 * (1.0 + np.sin(80.0 * np.pi * xc) * np.cos(80.0 * np.pi * yc)) * k_const
    return np.where(_fiveblock_mask(xc, yc), k_const, sinus)


def fiveblock_coarse_kappa_eq24(n: int = 40, k_const: float = 1.0, k_star: float = 8.485) -> np.ndarray:
    """Eq. 24: coarse ``kappa*`` on 40x40 points, ``k_const`` in the five blocks, else ``k_star * k_const``.

    The 1-based index ranges 19..22, 9..12 and 29..32 are the 0-based ranges
    18..21, 8..11 and 28..31.
    """
    idx = np.arange(n)

    def rng_(lo, hi):
        return (idx >= lo - 1) & (idx <= hi - 1)
    a = rng_(19, 22)[None, :] & rng_(19, 22)[:, None]
    b = rng_(9, 12)[None, :] & rng_(9, 12)[:, None]
    c = rng_(29, 32)[None, :] & rng_(29, 32)[:, None]
    d = rng_(9, 12)[None, :] & rng_(29, 32)[:, None]
    e = rng_(29, 32)[None, :] & rng_(9, 12)[:, None]
    return np.where(a | b | c | d | e, k_const, k_star * k_const).astype(np.float64)


def sinusoidal_g_field(n: int, g_scale: float, length: float = 1.0) -> np.ndarray:
    """Section 4.3.1: ``G = (sin(pi x), sin(pi y)) * g_scale`` at cell centres, shape ``[2, n, n]``."""
    dx = length / n
    c = (np.arange(n) + 0.5) * dx
    yc, xc = np.meshgrid(c, c, indexing="ij")
    return np.stack([np.sin(np.pi * xc), np.sin(np.pi * yc)]) * g_scale


def crop_periodic(a: np.ndarray, x0: int, y0: int, wx: int, wy: int) -> np.ndarray:
    """Window ``[y0, y0+wy) x [x0, x0+wx)`` of a periodic field, wrapping at the edges."""
    ny, nx = a.shape[-2:]
    rows = (np.arange(y0, y0 + wy) % ny)
    cols = (np.arange(x0, x0 + wx) % nx)
    return a[..., rows[:, None], cols[None, :]]
