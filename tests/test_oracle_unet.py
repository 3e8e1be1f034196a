"""Pins of the network reference (oracle/unet.py): the forward convolution
against scipy.signal.correlate, the data and weight gradients and the pooling
pair against finite differences / adjointness."""
import numpy as np
import pytest
import scipy.signal

from oracle import unet


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 4, 5, 6, 2))
    w = rng.standard_normal((3, 27, 2))
    y = unet.conv3d(x, w)
    for o in range(3):
        ref = np.zeros((4, 5, 6))
        for c in range(2):
            k = w[o, :, c].reshape(3, 3, 3)       # tap order (dt, dy, dx)
            ref += scipy.signal.correlate(x[0, :, :, :, c], k, mode="same")
        np.testing.assert_allclose(y[0, :, :, :, o], ref, atol=1e-12)


def _num_grad(f, a, eps=1e-6):
    g = np.zeros_like(a)
    it = np.nditer(a, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        a[i] += eps
        fp = f()
        a[i] -= 2 * eps
        fm = f()
        a[i] += eps
        g[i] = (fp - fm) / (2 * eps)
    return g


def test_conv3d_gradients_by_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 3, 3, 4, 2))
    w = rng.standard_normal((2, 27, 2))
    gy = rng.standard_normal((1, 3, 3, 4, 2))
    f = lambda: float(np.sum(unet.conv3d(x, w) * gy))
    np.testing.assert_allclose(unet.conv3d_dgrad(gy, w), _num_grad(f, x), atol=1e-6)
    np.testing.assert_allclose(unet.conv3d_wgrad(x, gy), _num_grad(f, w), atol=1e-6)


def test_pool_upsample_adjoint_pairs():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 4, 6, 3))
    g = rng.standard_normal((2, 3, 2, 3, 3))
    # <pool(x), g> = <x, pool_backward(g)>,  <upsample(g), x> = <g, upsample_backward(x)>
    assert np.sum(unet.pool(x) * g) == pytest.approx(np.sum(x * unet.pool_backward(g)), abs=1e-12)
    assert np.sum(unet.upsample(g) * x) == pytest.approx(np.sum(g * unet.upsample_backward(x)), abs=1e-12)
    np.testing.assert_allclose(unet.pool(unet.upsample(g)), g, atol=1e-15)


def test_mse_gradient():
    rng = np.random.default_rng(3)
    out = rng.standard_normal((2, 5))
    tgt = rng.standard_normal((2, 5))
    loss, g = unet.mse(out, tgt)
    np.testing.assert_allclose(g, _num_grad(lambda: unet.mse(out, tgt)[0], out), atol=1e-8)


def _net(widths, cin, cout, seed):
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co in unet.unet_layers(widths, cin, cout):
        params[name] = (rng.standard_normal((co, 27, ci)) * np.sqrt(2.0 / (27 * ci)), 0.1 * rng.standard_normal(co))
    return params


def test_adamw_closed_forms():
    """AdamW (Loshchilov and Hutter, decoupled weight decay) on cases whose update is known in closed form:
    with zero gradient only the decay acts, p (1 - lr wd); with a constant gradient the bias corrections make
    m_hat = g and v_hat = g^2 at every step, so each step moves p by -lr g / (|g| + eps) besides the decay."""
    lr, b1, b2, eps, wd = 1e-2, 0.9, 0.999, 1e-8, 0.1
    p0 = np.array([1.0, -2.0, 0.5])
    p, m, v = unet.adamw(p0.copy(), np.zeros(3), np.zeros(3), np.zeros(3), lr, b1, b2, eps, wd, 1)
    np.testing.assert_allclose(p, p0 * (1 - lr * wd), rtol=0, atol=1e-15)
    g = np.array([0.3, -4.0, 1e-3])
    p, m, v = p0.copy(), np.zeros(3), np.zeros(3)
    for step in range(1, 6):
        expect = p * (1 - lr * wd) - lr * g / (np.abs(g) + eps)
        p, m, v = unet.adamw(p, g, m, v, lr, b1, b2, eps, wd, step)
        np.testing.assert_allclose(p, expect, rtol=1e-12, atol=1e-15)


def test_round_bf16_against_the_format():
    # representable values stay, halfway cases go to the even neighbour, 1 + 2^-9 is below halfway
    assert unet.round_bf16(1.0) == 1.0
    assert unet.round_bf16(1.0 + 2.0 ** -8) == 1.0          # halfway between 1 and 1 + 2^-7, even is 1
    assert unet.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # halfway, even neighbour above
    assert unet.round_bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    assert unet.round_bf16(-3.0) == -3.0
    x = np.random.default_rng(5).standard_normal(1000)
    r = unet.round_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))


def test_unet_gradients_by_finite_differences():
    widths = (2, 3)
    params = _net(widths, 2, 2, 0)
    rng = np.random.default_rng(1)
    inp = rng.standard_normal((1, 2, 4, 4, 2))
    target = rng.standard_normal((1, 2, 4, 4, 1))
    loss, out, grads = unet.unet_forward_backward(params, widths, inp, target, 1)
    assert set(grads) == {n for n, _, _ in unet.unet_layers(widths, 2, 2)}
    eps = 1e-6
    for name, (w, b) in params.items():
        for arr, gidx in ((w, 0), (b, 1)):
            flat = arr.reshape(-1)
            for j in rng.choice(flat.size, size=min(4, flat.size), replace=False):
                old = flat[j]
                flat[j] = old + eps
                lp = unet.unet_forward_backward(params, widths, inp, target, 1)[0]
                flat[j] = old - eps
                lm = unet.unet_forward_backward(params, widths, inp, target, 1)[0]
                flat[j] = old
                num = (lp - lm) / (2 * eps)
                ana = grads[name][gidx].reshape(-1)[j]
                assert abs(num - ana) <= 1e-6 + 1e-5 * abs(num), (name, gidx, j, num, ana)
