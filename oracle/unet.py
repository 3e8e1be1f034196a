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


# ---------------------------------------------------------------------------
# The warm-start U-Net, composed from the layers above
# ---------------------------------------------------------------------------

def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    bfloat16 keeps the top 16 bits of an IEEE float32; rounding adds half of
    the dropped range (minus one when the kept part is even) before truncating.
    """
    f = np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unet_layers(widths, cin, cout):
    """(name, cin, cout) of every convolution, in forward order."""
    L = len(widths)
    out = []
    c = cin
    for l in range(L):
        out += [("e%da" % l, c, widths[l]), ("e%db" % l, widths[l], widths[l])]
        c = widths[l]
    for l in range(L - 2, -1, -1):
        out += [("d%da" % l, widths[l + 1] + widths[l], widths[l]), ("d%db" % l, widths[l], widths[l])]
    out.append(("head", widths[0], cout))
    return out


def unet_forward_backward(params, widths, inp, target, cv, rnd=None):
    """Loss, output and parameter gradients of the U-Net on one batch.

    Encoder level l: two ReLU convolutions, the second one's output s_l is the
    skip; 2 x 2 average pooling feeds level l + 1.  Decoder level l (deepest
    first): nearest upsampling of the deeper output, concatenated with s_l
    (upsampled channels first), then two ReLU convolutions.  A last linear
    convolution gives the output; the loss is the MSE over its first cv
    channels.  params[name] = (w [cout][27][cin], b [cout]).  ``rnd`` (e.g.
    round_bf16) is applied wherever a stored activation or activation gradient
    is rounded; weight gradients are not rounded.
    """
    R = rnd if rnd is not None else (lambda a: np.asarray(a, np.float64))
    L = len(widths)
    W = {k: (R(w), np.asarray(b, np.float64)) for k, (w, b) in params.items()}
    x = R(inp)
    acts = {}
    skips = []
    for l in range(L):
        a = R(conv3d(x, *W["e%da" % l], relu=True))
        s = R(conv3d(a, *W["e%db" % l], relu=True))
        acts["e%da" % l] = (x, a)
        acts["e%db" % l] = (a, s)
        skips.append(s)
        if l < L - 1:
            x = R(pool(s))
    h = skips[-1]
    for l in range(L - 2, -1, -1):
        c = np.concatenate([upsample(h), skips[l]], axis=-1)
        a = R(conv3d(c, *W["d%da" % l], relu=True))
        h2 = R(conv3d(a, *W["d%db" % l], relu=True))
        acts["d%da" % l] = (c, a)
        acts["d%db" % l] = (a, h2)
        h = h2
    out = conv3d(h, *W["head"])
    loss, gout = mse(out[..., :cv], target)
    g = np.zeros_like(out)
    g[..., :cv] = gout
    g = R(g)
    grads = {}

    def back(name, gy, need_dx=True):
        xin, y = acts[name] if name != "head" else (h, None)
        if y is not None:
            gy = relu_backward(gy, y)
        grads[name] = (conv3d_wgrad(xin, gy), gy.sum(axis=(0, 1, 2, 3)))
        return R(conv3d_dgrad(gy, W[name][0])) if need_dx else None

    gh = back("head", g)
    for l in range(L - 1):
        ga = back("d%db" % l, gh)
        gc = back("d%da" % l, ga)
        up_c = widths[l + 1]
        skip_grad_from_decoder = gc[..., up_c:]
        gh = R(upsample_backward(gc[..., :up_c]))
        skips[l] = (skips[l], skip_grad_from_decoder)
    gs = gh   # gradient of the deepest encoder output
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            gs = R(skips[l][1] + R(pool_backward(gx)))
        ga = back("e%db" % l, gs)
        gx = back("e%da" % l, ga, need_dx=l > 0)
    return loss, out, grads
