"""FP64 oracle of the learned K* surrogate -- TEST INFRASTRUCTURE ONLY.

The surrogate is an addition to the paper's method (the paper obtains every K*
from local LBM runs, Section 3). It maps a subdomain's permeability patch to
log K*_xx and log K*_yy; local LBM stays its fallback and the arbiter of its error.
This module restates what the library's kernels compute, plainly and in FP64,
so they can be checked: direct 3x3 'same' convolutions (one matmul per tap),
ReLU, global average pooling, a linear head, the backward pass of all of it,
the mean-squared-error loss, Adam, patch resampling and patch statistics.
Only tests, the smoke check and the benchmark's CPU baseline import it; it
shares no code with the CUDA path.

Layouts: activations [N, C, H, W]; conv weights [C_out, C_in, 3, 3]; head
weights [2, C]. Padding is zero padding of one cell on every side.
"""

from __future__ import annotations

import numpy as np

CHANNELS = (2, 32, 32, 64, 64, 64, 64)     # input planes: log kappa, leaf-size plane
PATCH = 32


# ---------------------------------------------------------------- patches

def resample_patch(logk: np.ndarray) -> np.ndarray:
    """A leaf's log-permeability (s x s) as a 32 x 32 patch.

    s < 32 (a divisor of 32): each cell is replicated (32 / s) x (32 / s) times;
    s = 32: unchanged; s > 32 (a multiple of 32): mean of log K over (s / 32)^2 blocks.
    """
    s = logk.shape[0]
    if s == PATCH:
        return logk.astype(np.float64).copy()
    if s < PATCH:
        if PATCH % s:
            raise ValueError("leaf size must divide 32")
        r = PATCH // s
        return np.repeat(np.repeat(logk, r, axis=0), r, axis=1).astype(np.float64)
    if s % PATCH:
        raise ValueError("leaf size must be a multiple of 32")
    r = s // PATCH
    return logk.reshape(PATCH, r, PATCH, r).mean(axis=(1, 3))


def patch_stats(p: np.ndarray) -> np.ndarray:
    """(mean, standard deviation, gradient energy) of a 32 x 32 log-K patch.

    Gradient energy: mean of squared forward differences along x and y over the
    patch interior (periodic differences are not used: a leaf is not periodic in K).
    """
    dx = p[:, 1:] - p[:, :-1]
    dy = p[1:, :] - p[:-1, :]
    ge = 0.5 * (np.mean(dx * dx) + np.mean(dy * dy))
    return np.array([p.mean(), p.std(), ge])


def make_input(logk_patch: np.ndarray, size: int, shift: float, scale: float) -> np.ndarray:
    """Two input planes: (log K - shift) / scale and the constant log2(size) / 6."""
    x = np.empty((2, PATCH, PATCH))
    x[0] = (logk_patch - shift) / scale
    x[1] = np.log2(size) / 6.0
    return x


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
            y += np.einsum("nchw,oc->nohw", win, w[:, :, dy, dx])
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
            dw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", dy, win)
            dxp[:, :, ky:ky + h, kx:kx + wd] += np.einsum("nohw,oc->nchw", dy, w[:, :, ky, kx])
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
