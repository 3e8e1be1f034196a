"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the transport method; it only draws
densities.  Both the CUDA path (through tests and the benchmark) and the FP64
oracle receive the same arrays from here.

* RGB pairs: per channel a sum of B Gaussian blobs (centres uniform over the
  image, standard deviation U[3, 6] pixels, amplitude U[0.5, 1]) plus a 1e-3
  floor, normalised to total mass 1 over pixels and channels.  f0 uses seed 2s
  and f1 seed 2s + 1 for pair s.  These stand in for the photographs of the
  paper's section 4, which are not available here.
* Hue pairs: a mixture of three von Mises bumps (concentration U[2, 20],
  uniform means, Dirichlet(1, 1, 1) weights) evaluated at the bin centres of n
  periodic bins and normalised to mass 1; they stand in for the hue histograms
  of section 5.
* Mixed batches: RGB sides from {64, 96, 128, 192, 256} with 16..48 time
  steps, hue pairs with 64..720 bins and 16..64 time steps.

Arrays are returned in the layout of the C ABI: RGB densities as
``[c][y][x]`` (shape (3, n2, n1)), hue histograms as ``[bin]``.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def rgb_blobs(n1: int, n2: int, nblobs: int, seed: int, C: int = 3,
              floor: float = 1e-3, dtype=np.float32) -> np.ndarray:
    """One RGB density of shape (C, n2, n1), mass 1 (see module docstring)."""
    rng = np.random.default_rng(seed)
    y = np.arange(n2, dtype=np.float64)[:, None] + 0.5
    x = np.arange(n1, dtype=np.float64)[None, :] + 0.5
    out = np.zeros((C, n2, n1), dtype=np.float64)
    for c in range(C):
        cx = rng.uniform(0.0, n1, nblobs)
        cy = rng.uniform(0.0, n2, nblobs)
        sd = rng.uniform(3.0, 6.0, nblobs)
        amp = rng.uniform(0.5, 1.0, nblobs)
        for b in range(nblobs):
            out[c] += amp[b] * np.exp(-((x - cx[b]) ** 2 + (y - cy[b]) ** 2) / (2.0 * sd[b] ** 2))
    out += floor
    out /= out.sum()
    return out.astype(dtype)


def rgb_pair(n1: int, n2: int, nblobs: int, s: int = 0, C: int = 3,
             dtype=np.float32) -> Tuple[np.ndarray, np.ndarray]:
    """Pair s: f0 from seed 2s, f1 from seed 2s+1; equal mass 1 (to rounding)."""
    f0 = rgb_blobs(n1, n2, nblobs, 2 * s, C, dtype=np.float64)
    f1 = rgb_blobs(n1, n2, nblobs, 2 * s + 1, C, dtype=np.float64)
    return f0.astype(dtype), f1.astype(dtype)


def hue_hist(nbins: int, seed: int, nbumps: int = 3, dtype=np.float32) -> np.ndarray:
    """Von Mises mixture on the circle binned to nbins bins, mass 1."""
    rng = np.random.default_rng(seed)
    kappa = rng.uniform(2.0, 20.0, nbumps)
    mu = rng.uniform(0.0, 2.0 * np.pi, nbumps)
    w = rng.dirichlet(np.ones(nbumps))
    theta = (np.arange(nbins, dtype=np.float64) + 0.5) * (2.0 * np.pi / nbins)
    h = np.zeros(nbins)
    for j in range(nbumps):
        h += w[j] * np.exp(kappa[j] * (np.cos(theta - mu[j]) - 1.0))
    h /= h.sum()
    return h.astype(dtype)


def hue_pair(nbins: int, s: int = 0, dtype=np.float32) -> Tuple[np.ndarray, np.ndarray]:
    h0 = hue_hist(nbins, 2 * s, dtype=np.float64)
    h1 = hue_hist(nbins, 2 * s + 1, dtype=np.float64)
    return h0.astype(dtype), h1.astype(dtype)


def mixed_batch(seed: int = 0, n_rgb: int = 16, n_hue: int = 64) -> Tuple[List[dict], List[dict]]:
    """Descriptors of the mixed batch: RGB and hue problem sizes with pair seeds."""
    rng = np.random.default_rng(seed)
    sides = [64, 96, 128, 192, 256]
    rgb = []
    for i in range(n_rgb):
        n1 = int(rng.choice(sides))
        n2 = int(rng.choice(sides))
        P = int(rng.integers(16, 49))
        rgb.append({"n1": n1, "n2": n2, "P": P, "s": 1000 + i})
    hue = []
    for i in range(n_hue):
        hue.append({"n": int(rng.integers(64, 721)), "P": int(rng.integers(16, 65)), "s": 2000 + i})
    return rgb, hue


def hue_image_pair(n: int, seed: int = 0, dtype=np.float32) -> Tuple[np.ndarray, np.ndarray]:
    """Two n x n RGB images ([3][n][n] in [0, 1]) with the same saturation and value that differ only in
    hue, like the yellow and red flowers of section 5: a flower (a union of Gaussian petals) on a green
    background.  Every pixel has max channel V and min channel V (1 - S); the third channel sets the hue
    inside the sector: between red and yellow in the flower (yellow-orange in the first image, red-orange
    in the second), between green and cyan-green in the background."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:n, 0:n] + 0.5
    flower = np.zeros((n, n))
    for _ in range(6):
        cx, cy = rng.uniform(0.3, 0.7, 2) * n
        r = rng.uniform(0.06, 0.14) * n
        flower = np.maximum(flower, np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * r * r)))
    inside = flower > 0.5
    V = 0.35 + 0.6 * (0.5 + 0.5 * np.sin(2 * np.pi * (xx / n * rng.uniform(1, 3) + rng.uniform())))
    S = 0.4 + 0.5 * flower
    w = np.clip(0.5 + 0.15 * rng.standard_normal((n, n)), 0, 1)       # position inside the sector
    lo = V * (1 - S)
    imgs = []
    for warm in (0.85, 0.12):
        mid = lo + (V - lo) * np.where(inside, np.clip(warm + 0.1 * (w - 0.5), 0, 1), 0.3 * w)
        r = np.where(inside, V, lo)
        g = np.where(inside, mid, V)
        b = np.where(inside, lo, mid)
        imgs.append(np.stack([r, g, b]).astype(dtype))
    return imgs[0], imgs[1]
