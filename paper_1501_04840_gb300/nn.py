"""ctypes binding of the warm-start network kernels (ot_nn_* in include/dynot.h).

Argument marshalling only: every operation runs in libdynot.so on the caller's
CUDA stream.  Activations are channel slices of channels-last bf16 buffers
[N][T][Y][X][C]; a slice is (buffer, first channel, channel count).
"""
from __future__ import annotations

import ctypes
from ctypes import c_float, c_int, c_longlong, c_void_p
from dataclasses import dataclass

import torch

from .binding import _check, load_library

_nn = None


def lib():
    global _nn
    if _nn is not None:
        return _nn
    L = load_library()
    vp, i, ll, f = c_void_p, c_int, c_longlong, c_float
    sig = {
        "ot_nn_conv3d": [i, i, i, i, i, i, vp, i, i, vp, vp, vp, i, i, i, i, vp],
        "ot_nn_conv3d_wgrad": [i, i, i, i, i, i, vp, i, i, vp, i, i, vp, vp, vp],
        "ot_nn_rotate_weights": [i, i, vp, vp, vp],
        "ot_nn_relu_grad": [ll, i, vp, i, i, vp, i, i, vp],
        "ot_nn_pool": [i, i, i, i, i, vp, i, i, vp, i, i, i, vp],
        "ot_nn_upsample": [i, i, i, i, i, vp, i, i, vp, i, i, i, vp],
        "ot_nn_add_slice": [ll, i, vp, i, i, vp, i, i, vp],
        "ot_nn_mse": [ll, i, vp, i, vp, vp, i, vp, vp],
        "ot_nn_adamw": [ll, vp, vp, vp, vp, vp, f, f, f, f, f, i, vp],
        "ot_nn_to_bf16": [ll, vp, vp, vp],
        "ot_nn_make_input": [i, i, i, i, i, vp, vp, vp, vp, vp],
        "ot_nn_path_channels": [i, i, i, i, i, vp, vp, vp, vp, vp, i, vp],
        "ot_nn_dual_channels": [i, i, i, i, i, vp, vp, i, i, vp],
        "ot_nn_check": [vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = c_int
    _nn = L
    return L


def _p(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise TypeError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _s(stream):
    return None if stream is None else ctypes.c_void_p(stream.cuda_stream)


@dataclass
class Slice:
    """Channels [off, off + C) of the channels-last buffer `buf` (last dim = its channel stride)."""
    buf: torch.Tensor
    off: int
    C: int

    @property
    def stride(self) -> int:
        return self.buf.shape[-1]

    @property
    def voxels(self) -> int:
        return self.buf.numel() // self.buf.shape[-1]


def whole(buf: torch.Tensor) -> Slice:
    return Slice(buf, 0, buf.shape[-1])


def conv3d(vol, x: Slice, w, bias, y: Slice, relu: bool, out_f32: bool = False, stream=None):
    N, T, Y, X = vol
    _check(lib().ot_nn_conv3d(N, T, Y, X, x.C, y.C, _p(x.buf), x.stride, x.off, _p(w), _p(bias), _p(y.buf),
                              y.stride, y.off, int(relu), int(out_f32), _s(stream)))


def conv3d_wgrad(vol, x: Slice, dy: Slice, dw, db, stream=None):
    N, T, Y, X = vol
    _check(lib().ot_nn_conv3d_wgrad(N, T, Y, X, x.C, dy.C, _p(x.buf), x.stride, x.off, _p(dy.buf), dy.stride,
                                    dy.off, _p(dw), _p(db), _s(stream)))


def rotate_weights(cin: int, cout: int, w, wr, stream=None):
    _check(lib().ot_nn_rotate_weights(cin, cout, _p(w), _p(wr), _s(stream)))


def relu_grad(g: Slice, y: Slice, stream=None):
    _check(lib().ot_nn_relu_grad(g.voxels, g.C, _p(g.buf), g.stride, g.off, _p(y.buf), y.stride, y.off,
                                 _s(stream)))


def pool(vol_coarse, x: Slice, y: Slice, backward: bool = False, stream=None):
    N, T, Yc, Xc = vol_coarse
    _check(lib().ot_nn_pool(N, T, Yc, Xc, x.C, _p(x.buf), x.stride, x.off, _p(y.buf), y.stride, y.off,
                            int(backward), _s(stream)))


def upsample(vol_coarse, x: Slice, y: Slice, backward: bool = False, stream=None):
    N, T, Yc, Xc = vol_coarse
    _check(lib().ot_nn_upsample(N, T, Yc, Xc, x.C, _p(x.buf), x.stride, x.off, _p(y.buf), y.stride, y.off,
                                int(backward), _s(stream)))


def add_slice(x: Slice, y: Slice, stream=None):
    _check(lib().ot_nn_add_slice(x.voxels, x.C, _p(x.buf), x.stride, x.off, _p(y.buf), y.stride, y.off,
                                 _s(stream)))


def mse(out, cv: int, target, g, loss, stream=None):
    """out: fp32 [M][os]; target bf16 [M][cv]; g bf16 [M][gs]; loss fp32 [1] (accumulated)."""
    M = target.numel() // cv
    _check(lib().ot_nn_mse(M, cv, _p(out), out.shape[-1], _p(target), _p(g), g.shape[-1], _p(loss), _s(stream)))


def adamw(p, g, m, v, pb, lr, b1, b2, eps, wd, step, stream=None):
    _check(lib().ot_nn_adamw(p.numel(), _p(p), _p(g), _p(m), _p(v), _p(pb), lr, b1, b2, eps, wd, step,
                             _s(stream)))


def to_bf16(x, y, stream=None):
    _check(lib().ot_nn_to_bf16(x.numel(), _p(x), _p(y), _s(stream)))


def make_input(N, P, Y, X, f0, f1, out, scale=None, stream=None):
    _check(lib().ot_nn_make_input(N, P, Y, X, out.shape[-1], _p(f0), _p(f1), _p(scale), _p(out), _s(stream)))


def path_channels(N, Y, X, P, to_channels: bool, packed, ch, f0=None, f1=None, scale=None, stream=None):
    _check(lib().ot_nn_path_channels(N, Y, X, P, int(to_channels), _p(scale), _p(f0), _p(f1), _p(packed), _p(ch),
                                     ch.shape[-1], _s(stream)))


def dual_channels(N, Y, X, P, to_channels: bool, packed, ch, co: int, stream=None):
    _check(lib().ot_nn_dual_channels(N, Y, X, P, int(to_channels), _p(packed), _p(ch), ch.shape[-1], co,
                                     _s(stream)))


def check(stream=None):
    """ot_nn_check: wait for the stream and raise if a bounded device wait of the tcgen05 convolution ran
    out since the last check."""
    _check(lib().ot_nn_check(_s(stream)))
