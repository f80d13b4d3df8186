"""FP64 oracle of the learned K* surrogate -- TEST INFRASTRUCTURE ONLY.

The surrogate is an addition to the paper's method (the paper obtains every K*
from local LBM runs, Section 3). It maps a subdomain's permeability patch to
log K*_xx and log K*_yy; local LBM stays its fallback and the arbiter of its error.
This module restates what the library's kernels compute, plainly and in FP64,
so they can be checked: direct 3x3 'same' convolutions (one matmul per tap),
ReLU, global average pooling, a linear head, the backward pass of all of it,
the mean-squared-error loss, Adam, the leaf-to-input planes, patch statistics,
the per-leaf target base and the gate that accepts a prediction or sends the
leaf back to local LBM.
Only tests, the smoke check and the benchmark's CPU baseline import it; it
shares no code with the CUDA path.

Layouts: activations [N, C, H, W]; conv weights [C_out, C_in, 3, 3]; head
weights [2, C]. Padding is zero padding of one cell on every side.
"""

from __future__ import annotations

import numpy as np

CHANNELS = (9, 32, 32, 64, 64, 64, 64)     # input planes: 4 phase planes, size plane, 4 context planes
PATCH = 32
PHASES = 4


# ---------------------------------------------------------------- patches

def _check_size(s: int) -> None:
    if not ((1 <= s <= PATCH and PATCH % s == 0) or (s % 64 == 0 and 64 <= s <= 1024)):
        raise ValueError("leaf size must divide 32 or be a multiple of 64 up to 1024")


def full_plane(logk: np.ndarray) -> np.ndarray:
    """A leaf's log-permeability (s x s) on a 64 x 64 plane.

    s < 64 (a divisor of 32): each cell repeated (64 / s) x (64 / s) times;
    s = 64: the leaf itself; s = 64 r (r >= 2): the mean of log K over r x r blocks.
    """
    s = logk.shape[0]
    _check_size(s)
    if s < 64:
        r = 64 // s
        return np.repeat(np.repeat(logk, r, axis=0), r, axis=1).astype(np.float64)
    r = s // 64
    return logk.astype(np.float64).reshape(64, r, 64, r).mean(axis=(1, 3))


def phase_planes(logk: np.ndarray) -> np.ndarray:
    """The 64 x 64 plane of full_plane split by the parity of its row and column:
    plane 2 a + b holds cell (2 i + a, 2 j + b) at (i, j), so the four 32 x 32 planes carry
    every cell of a 64-cell leaf (and four equal copies of a leaf of 32 cells or fewer)."""
    f = full_plane(logk)
    return np.stack([f[a::2, b::2] for a in (0, 1) for b in (0, 1)])


def resample_patch(logk: np.ndarray) -> np.ndarray:
    """A leaf's log-permeability as one 32 x 32 patch: the mean of its four phase planes
    (the leaf repeated for s <= 32; 2 x 2 block means of log K for s = 64)."""
    return phase_planes(logk).mean(axis=0)


def patch_stats(p: np.ndarray) -> np.ndarray:
    """(mean, standard deviation, gradient energy) of a 32 x 32 log-K patch.

    Gradient energy: mean of squared forward differences along x and y over the
    patch interior (periodic differences are not used: a leaf is not periodic in K).
    """
    dx = p[:, 1:] - p[:, :-1]
    dy = p[1:, :] - p[:-1, :]
    ge = 0.5 * (np.mean(dx * dx) + np.mean(dy * dy))
    return np.array([p.mean(), p.std(), ge])


def context_planes(p: np.ndarray) -> np.ndarray:
    """Four 32 x 32 planes of row and column means of K = exp(p) over a 32 x 32 log-K patch p, in
    log K: the harmonic and the arithmetic mean along x of each row (the same value across the
    row), then the harmonic and the arithmetic mean along y of each column (the same value down
    the column). These are the series and parallel means the layered arrangements are made of."""
    k = np.exp(np.asarray(p, dtype=np.float64))
    hx = -np.log(np.mean(1.0 / k, axis=1))
    ax = np.log(np.mean(k, axis=1))
    hy = -np.log(np.mean(1.0 / k, axis=0))
    ay = np.log(np.mean(k, axis=0))
    n = k.shape[0]
    return np.stack([np.repeat(hx[:, None], n, axis=1), np.repeat(ax[:, None], n, axis=1),
                     np.repeat(hy[None, :], n, axis=0), np.repeat(ay[None, :], n, axis=0)])


def make_input(logk: np.ndarray, shift: float, scale: float) -> np.ndarray:
    """Nine input planes of a leaf: its four phase planes as (log K - shift) / scale, the
    constant log2(size) / 6, and the four context planes of its 32 x 32 patch (resample_patch),
    also as (log K - shift) / scale."""
    x = np.empty((9, PATCH, PATCH))
    ph = phase_planes(logk)
    x[:4] = (ph - shift) / scale
    x[4] = np.log2(logk.shape[0]) / 6.0
    x[5:] = (context_planes(ph.mean(axis=0)) - shift) / scale
    return x


def layered_bounds(k: np.ndarray):
    """Bounds on the effective permeability of a rectangular patch k [rows = y][columns = x]
    from two layered arrangements (the series and parallel means of Tables 1 and 2).

    Flow along x: the rows taken as separate tubes in parallel, each the series (harmonic)
    mean of its cells, give the lower value lo_x = mean over rows of H_x; the columns taken as
    slabs in series, each the parallel (arithmetic) mean of its cells, give the upper value
    hi_x = harmonic mean over columns of A_y. Flow along y: the same with rows and columns
    exchanged. Returns (lo_x, hi_x, lo_y, hi_y).
    """
    k = np.asarray(k, dtype=np.float64)
    h_rows = 1.0 / np.mean(1.0 / k, axis=1)          # H_x of each row
    a_cols = np.mean(k, axis=0)                      # A_y of each column
    h_cols = 1.0 / np.mean(1.0 / k, axis=0)          # H_y of each column
    a_rows = np.mean(k, axis=1)                      # A_x of each row
    return (np.mean(h_rows), 1.0 / np.mean(1.0 / a_cols),
            np.mean(h_cols), 1.0 / np.mean(1.0 / a_rows))


def darcy_solve(k: np.ndarray, drive: int):
    """Darcy flow through a periodic patch k [rows = y][columns = x] by finite volumes: the flux
    across the face between two neighbouring cells is k_f (p_i - p_j + G . (x_j - x_i)) with k_f the
    harmonic mean of the two cells, every cell conserves mass, and a unit force G drives the flow
    along x (drive 0) or y (drive 1). Solved by a sparse direct solve with one pressure fixed, then
    shifted to zero mean (the pressure is defined up to a constant). Returns (p, qx, qy): the
    pressure and the fluxes across each cell's +x and +y faces."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    k = np.asarray(k, dtype=np.float64)
    n_y, n_x = k.shape
    cells = n_x * n_y
    idx = np.arange(cells).reshape(n_y, n_x)
    faces = []                                            # (neighbour index, face permeability, axis)
    for axis in (1, 0):
        kn = np.roll(k, -1, axis=axis)
        faces.append((np.roll(idx, -1, axis=axis).ravel(), (2.0 * k * kn / (k + kn)).ravel(), axis))
    i = idx.ravel()
    rows, cols, vals = [], [], []
    for j, kf, _ in faces:
        rows += [i, i, j, j]
        cols += [i, j, j, i]
        vals += [kf, -kf, kf, -kf]
    a = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(cells, cells))
    a = (a + sp.csr_matrix(([1.0], ([0], [0])), shape=(cells, cells))).tocsc()
    axis_d = 1 if drive == 0 else 0
    b = np.zeros(cells)
    for j, kf, axis in faces:
        if axis == axis_d:                                # the force pushes flux from i to j
            np.add.at(b, i, -kf)
            np.add.at(b, j, kf)
    p = sla.spsolve(a, b)
    p -= p.mean()
    q = []
    for j, kf, axis in faces:
        q.append((kf * (p[i] - p[j] + (1.0 if axis == axis_d else 0.0))).reshape(n_y, n_x))
    return p.reshape(n_y, n_x), q[0], q[1]


def darcy_keff(k: np.ndarray):
    """Effective permeability (K*_xx, K*_yy) of a periodic patch under Darcy's law by finite
    volumes (darcy_solve): K* along the drive is the mean face flux per unit force (unit
    viscosity)."""
    _, qx, _ = darcy_solve(k, 0)
    _, _, qy = darcy_solve(k, 1)
    return float(np.mean(qx)), float(np.mean(qy))


def target_base(logk: np.ndarray, mode: int):
    """Per-leaf base (c_xx, w_xx, c_yy, w_yy) of the surrogate's target: the networks learn
    (log K* - c) / w for each component.

    mode 0: c = mean log K of the leaf's 64 x 64 plane, w = 1;
    mode 1: c = midpoint of log lo and log hi of layered_bounds on that plane, w = 1;
    mode 2: the same c and w = max((log hi - log lo) / 2, 0.05);
    mode 3: c = log of darcy_keff on the leaf itself (its 64 x 64 plane above 64 cells), w = 1.
    """
    if mode == 3:
        leaf = logk if logk.shape[0] <= 64 else full_plane(logk)
        kxx, kyy = darcy_keff(np.exp(np.asarray(leaf, dtype=np.float64)))
        return (np.log(kxx), 1.0, np.log(kyy), 1.0)
    f = full_plane(logk)
    if mode == 0:
        m = f.mean()
        return (m, 1.0, m, 1.0)
    lox, hix, loy, hiy = (np.log(v) for v in layered_bounds(np.exp(f)))
    wx = 1.0 if mode == 1 else max(0.5 * (hix - lox), 0.05)
    wy = 1.0 if mode == 1 else max(0.5 * (hiy - loy), 0.05)
    return (0.5 * (lox + hix), wx, 0.5 * (loy + hiy), wy)


# ---------------------------------------------------------------- the gate

def gate(y: np.ndarray, stats: np.ndarray, sizes: np.ndarray, stat_lo, stat_hi, spread_max):
    """Which leaves take the ensemble's prediction and which go back to local LBM.

    y [M][n][2]: log K*_xx and log K*_yy of each of the M members; stats [n][3] the patch
    statistics; sizes [n] the leaf sizes; stat_lo, stat_hi [3] the accepted range of each
    statistic (bounds included); spread_max a relative spread, or a mapping from leaf size to
    one. Leaf i is accepted when, for both components, the members' sample standard deviation
    (denominator M - 1; 0 for one member) is at most ln(1 + spread_max) and their mean is
    finite, and every statistic lies in its range. Returns (accept [n] bool, keff [n][4]):
    keff = (exp(mean xx), 0, 0, exp(mean yy)) for accepted leaves, NaN for the others.
    """
    y = np.asarray(y, dtype=np.float64)
    m_members, n, _ = y.shape
    accept = np.zeros(n, dtype=bool)
    keff = np.full((n, 4), np.nan)
    for i in range(n):
        smax = spread_max[int(sizes[i])] if isinstance(spread_max, dict) else spread_max
        thr = np.log1p(smax)
        ok = True
        mean = np.zeros(2)
        for c in range(2):
            v = y[:, i, c]
            mean[c] = v.sum() / m_members
            sd = np.sqrt(((v - mean[c]) ** 2).sum() / (m_members - 1)) if m_members > 1 else 0.0
            if not (sd <= thr) or not np.isfinite(mean[c]):
                ok = False
        for k in range(3):
            if not (stat_lo[k] <= stats[i, k] <= stat_hi[k]):
                ok = False
        accept[i] = ok
        if ok:
            keff[i] = (np.exp(mean[0]), 0.0, 0.0, np.exp(mean[1]))
    return accept, keff


# ---------------------------------------------------------------- network

def init_params(seed: int, channels=CHANNELS) -> dict:
    """He-normal conv weights, zero biases, small head (seeded PCG64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        p[f"w{l}"] = rng.standard_normal((co, ci, 3, 3)) * np.sqrt(2.0 / (9 * ci))
        p[f"b{l}"] = np.zeros(co)
    c = channels[-1]
    p["wh"] = rng.standard_normal((2, c)) * np.sqrt(1.0 / c)
    p["bh"] = np.zeros(2)
    return p


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n, o, i, j] = b[o] + sum_{c, dy, dx} w[o, c, dy, dx] x[n, c, i + dy - 1, j + dx - 1] (zero padded)."""
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((n, w.shape[0], h, wd))
    for dy in range(3):
        for dx in range(3):
            win = xp[:, :, dy:dy + h, dx:dx + wd]                     # [n, c, h, w]
            y += np.einsum("nchw,oc->nohw", win, w[:, :, dy, dx], optimize=True)
    return y + b[None, :, None, None]


def conv3x3_backward(x, w, dy):
    """Gradients of conv3x3 w.r.t. its input, weights and bias given dL/dy."""
    n, c, h, wd = x.shape
    xp = np.zeros((n, c, h + 2, wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            win = xp[:, :, ky:ky + h, kx:kx + wd]
            dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", dy, win, optimize=True)
            dxp[:, :, ky:ky + h, kx:kx + wd] += np.einsum("nohw,oc->nchw", dy, w[:, :, ky, kx], optimize=True)
    db = dy.sum(axis=(0, 2, 3))
    return dxp[:, :, 1:-1, 1:-1], dw, db


def forward(p: dict, x: np.ndarray, nlayers: int = 6):
    """Returns (prediction [N, 2], cache) for inputs x [N, 2, 32, 32]."""
    acts = [x]
    h = x
    for l in range(nlayers):
        h = np.maximum(conv3x3(h, p[f"w{l}"], p[f"b{l}"]), 0.0)
        acts.append(h)
    pooled = h.mean(axis=(2, 3))                                       # [N, C]
    y = pooled @ p["wh"].T + p["bh"]
    return y, (acts, pooled)


def backward(p: dict, cache, dy: np.ndarray, nlayers: int = 6) -> dict:
    acts, pooled = cache
    g = {"wh": dy.T @ pooled, "bh": dy.sum(axis=0)}
    dpool = dy @ p["wh"]                                               # [N, C]
    h = acts[-1]
    dh = np.broadcast_to(dpool[:, :, None, None] / (h.shape[2] * h.shape[3]), h.shape).copy()
    for l in reversed(range(nlayers)):
        dh = dh * (acts[l + 1] > 0.0)                                  # ReLU
        dx, dw, db = conv3x3_backward(acts[l], p[f"w{l}"], dh)
        g[f"w{l}"], g[f"b{l}"] = dw, db
        dh = dx
    return g


def mse(y: np.ndarray, t: np.ndarray):
    """Loss mean((y - t)^2) over all entries and its gradient."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def adam_step(param, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): returns the new (param, m, v); t counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v
