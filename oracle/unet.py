"""FP64 reference of the warm-start network's layers.

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA network kernels.
The paper has no network; these are the textbook definitions of the layers
the warm start uses, written out in numpy (channels-last arrays
[n][t][y][x][c], weights [cout][27][cin] with tap = 9 (dt+1) + 3 (dy+1) + (dx+1)).
Pins: tests/test_oracle_unet.py (scipy.signal.correlate for the forward
convolution, finite differences for both gradients and the pooling pair).
"""
from __future__ import annotations

import numpy as np

TAPS = [(dt, dy, dx) for dt in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _pad(x):
    return np.pad(x, [(0, 0), (1, 1), (1, 1), (1, 1), (0, 0)])


def conv3d(x, w, b=None, relu=False):
    """y[v, o] = sum_tap sum_c w[o, tap, c] x[v + tap, c] (+ b[o]), zero padding."""
    N, T, Y, X, _ = x.shape
    xp = _pad(np.asarray(x, np.float64))
    y = np.zeros((N, T, Y, X, w.shape[0]))
    for k, (dt, dy, dx) in enumerate(TAPS):
        win = xp[:, 1 + dt:1 + dt + T, 1 + dy:1 + dy + Y, 1 + dx:1 + dx + X, :]
        y += np.einsum("ntyxc,oc->ntyxo", win, np.asarray(w[:, k, :], np.float64))
    if b is not None:
        y += np.asarray(b, np.float64)
    return np.maximum(y, 0.0) if relu else y


def conv3d_dgrad(dy, w):
    """dx[v, c] = sum_tap sum_o dy[v - tap, o] w[o, tap, c]."""
    N, T, Y, X, _ = dy.shape
    gp = _pad(np.asarray(dy, np.float64))
    dx = np.zeros((N, T, Y, X, w.shape[2]))
    for k, (dt, ddy, dxx) in enumerate(TAPS):
        win = gp[:, 1 - dt:1 - dt + T, 1 - ddy:1 - ddy + Y, 1 - dxx:1 - dxx + X, :]
        dx += np.einsum("ntyxo,oc->ntyxc", win, np.asarray(w[:, k, :], np.float64))
    return dx


def conv3d_wgrad(x, dy):
    """dw[o, tap, c] = sum_v dy[v, o] x[v + tap, c]."""
    N, T, Y, X, C = x.shape
    xp = _pad(np.asarray(x, np.float64))
    g = np.asarray(dy, np.float64)
    dw = np.zeros((g.shape[4], 27, C))
    for k, (dt, ddy, dxx) in enumerate(TAPS):
        win = xp[:, 1 + dt:1 + dt + T, 1 + ddy:1 + ddy + Y, 1 + dxx:1 + dxx + X, :]
        dw[:, k, :] = np.einsum("ntyxo,ntyxc->oc", g, win)
    return dw


def pool(x):
    """2 x 2 average pooling over (y, x)."""
    N, T, Y, X, C = x.shape
    return np.asarray(x, np.float64).reshape(N, T, Y // 2, 2, X // 2, 2, C).mean(axis=(3, 5))


def pool_backward(g):
    return np.repeat(np.repeat(np.asarray(g, np.float64), 2, axis=2), 2, axis=3) * 0.25


def upsample(x):
    """Nearest-neighbour 2x upsampling over (y, x)."""
    return np.repeat(np.repeat(np.asarray(x, np.float64), 2, axis=2), 2, axis=3)


def upsample_backward(g):
    N, T, Y, X, C = g.shape
    return np.asarray(g, np.float64).reshape(N, T, Y // 2, 2, X // 2, 2, C).sum(axis=(3, 5))


def relu_backward(g, y):
    return np.where(np.asarray(y) > 0, g, 0.0)


def mse(out, target):
    """loss = mean((out - target)^2), gradient 2 (out - target) / count."""
    d = np.asarray(out, np.float64) - np.asarray(target, np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def adamw(p, g, m, v, lr, b1, b2, eps, wd, step):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p * (1 - lr * wd) - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return p, m, v
