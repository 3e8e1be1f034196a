"""Hue image pipeline of section 5 over the C ABI (argument marshalling only).

Two images that differ only in hue are morphed into each other: their hue
histograms are transported with the periodic optimal transport of the paper
(a hue plan, Algorithm 1), and each intermediate histogram h^t becomes an
image u_t by specifying the source's hues to it, keeping the source's
saturation and value.  Every step runs in libdynot.so on the current torch
stream.
"""
from __future__ import annotations

import ctypes
from ctypes import c_int, c_void_p
from typing import List

import numpy as np
import torch

from .binding import Plan, _check, hue_grid, load_library

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = load_library()
        L.ot_rgb_to_hsv.argtypes = [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.ot_hsv_to_rgb.argtypes = [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]
        L.ot_hue_histogram.argtypes = [c_int, c_void_p, c_int, c_void_p, c_void_p]
        L.ot_hue_specify.argtypes = [c_int, c_void_p, c_int, c_void_p, c_void_p, c_void_p]
        for f in (L.ot_rgb_to_hsv, L.ot_hsv_to_rgb, L.ot_hue_histogram, L.ot_hue_specify):
            f.restype = c_int
        _lib = L
    return _lib


def _p(t: torch.Tensor):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return t.data_ptr()


def _s():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def rgb_to_hsv(rgb: torch.Tensor):
    """rgb [3][...] -> (h, s, v), each of the pixel shape."""
    n = rgb[0].numel()
    h, s, v = (torch.empty(rgb.shape[1:], dtype=torch.float32, device=rgb.device) for _ in range(3))
    _check(lib().ot_rgb_to_hsv(n, _p(rgb), _p(h), _p(s), _p(v), _s()))
    return h, s, v


def hsv_to_rgb(h: torch.Tensor, s: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    rgb = torch.empty((3,) + tuple(h.shape), dtype=torch.float32, device=h.device)
    _check(lib().ot_hsv_to_rgb(h.numel(), _p(h), _p(s), _p(v), _p(rgb), _s()))
    return rgb


def hue_histogram(h: torch.Tensor, bins: int) -> torch.Tensor:
    hist = torch.empty(bins, dtype=torch.float32, device=h.device)
    _check(lib().ot_hue_histogram(h.numel(), _p(h), bins, _p(hist), _s()))
    return hist


def specify(h: torch.Tensor, bins: int, target: torch.Tensor) -> torch.Tensor:
    out = torch.empty_like(h)
    _check(lib().ot_hue_specify(h.numel(), _p(h), bins, _p(target), _p(out), _s()))
    return out


def hue_morph(rgb0, rgb1, bins: int = 360, P: int = 16, iters: int = 5000, tol: float = 1e-5, device="cuda"):
    """Frames u_t, t = k / P (k = 0..P), of the hue transport between two images with the same saturation
    and value ([3][H][W] arrays in [0, 1]).  Returns (frames [P + 1][3][H][W], histogram path [P + 1][bins],
    solver stats)."""
    rgb0 = torch.as_tensor(np.ascontiguousarray(rgb0, np.float32)).to(device)
    rgb1 = torch.as_tensor(np.ascontiguousarray(rgb1, np.float32)).to(device)
    h0, s0, v0 = rgb_to_hsv(rgb0)
    h1, _, _ = rgb_to_hsv(rgb1)
    f0, f1 = hue_histogram(h0, bins), hue_histogram(h1, bins)
    plan = Plan(hue_grid(bins, P), stream=torch.cuda.current_stream().cuda_stream or None)
    torch.cuda.current_stream().synchronize()
    st = plan.solve(f0, f1, iters, tol)
    path = plan.path(out="torch", device=device)["f"][0]          # [P - 1][bins], interior times
    plan.close()
    hists: List[torch.Tensor] = [f0] + [path[k].contiguous() for k in range(P - 1)] + [f1]
    frames = [hsv_to_rgb(specify(h0, bins, ht), s0, v0) for ht in hists]
    return torch.stack(frames), torch.stack(hists), st
