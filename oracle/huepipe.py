"""Reference of the hue image pipeline of section 5 (numpy, float64).

TEST INFRASTRUCTURE ONLY: used by tests/ to check the CUDA pipeline kernels.

Section 5 transports the hue histogram of an image into another one with the
periodic OT of the paper and turns each intermediate histogram h^t back into
an image by histogram specification of the source hues, keeping saturation
and value.  The steps, as written here:

* HSV of an RGB pixel: the hexcone model (V = max, S = (max - min) / max,
  hue in [0, 1) from the sector of the largest channel); pinned against
  Python's colorsys.
* Hue histogram: pixel counts in `bins` equal bins of [0, 1), normalised to
  mass 1 (the empirical density of section 5).
* Periodic exact histogram specification (the paper cites an analysis of
  circular transport and an exact specification method without printing
  either; this is the reading used):
  - pixels are ranked by a strict order, (hue quantised to 32 bits, pixel
    index), so that every pixel has its own rank;
  - the target histogram becomes exact integer counts (largest remainders,
    ties to the lower bin);
  - the circle is cut where the squared circular distance (the cost of the
    paper's transport) is least: with the source hues sorted, x_r, and the
    target hues of the exact counts sorted, y_q, a shift s assigns rank r the
    target rank (r - s) mod npix at cost sum_r d(x_r, y_{(r-s) mod npix})^2,
    d the distance on the circle of circumference 1, and s is the minimiser
    over all npix shifts (ties to the smaller shift);
  - target rank q inside bin b (cumulative count C_b, count c_b) gets the hue
    (b + (q - C_b + 1/2) / c_b) / bins.
  Pinned: the output histogram equals the target counts exactly; the source's
  own histogram keeps every pixel in its bin; a target rotated by up to three bins
  moves every pixel by that rotation (either way, across the seam); the best
  cyclic shift reaches the optimal assignment over all permutations (Hungarian
  method) on small inputs; a single bump rotated by k bins on 4096 and more
  pixels is cut at the rotation, whose shift and cost are known in closed form.
"""
from __future__ import annotations

import numpy as np


def rgb_to_hsv(rgb):
    """rgb: [3][npix] in [0, 1] -> (h, s, v), hue in [0, 1)."""
    r, g, b = (np.asarray(c, np.float64) for c in rgb)
    mx = np.maximum(np.maximum(r, g), b)
    mn = np.minimum(np.minimum(r, g), b)
    d = mx - mn
    v = mx
    s = np.where(mx > 0, d / np.where(mx > 0, mx, 1.0), 0.0)
    safe = np.where(d > 0, d, 1.0)
    h = np.where(mx == r, ((g - b) / safe) % 6.0,
                 np.where(mx == g, (b - r) / safe + 2.0, (r - g) / safe + 4.0))
    h = np.where(d > 0, h / 6.0, 0.0)
    h = np.where(h >= 1.0, h - 1.0, h)
    return h, s, v


def hsv_to_rgb(h, s, v):
    h = np.asarray(h, np.float64)
    s = np.asarray(s, np.float64)
    v = np.asarray(v, np.float64)
    h6 = h * 6.0
    i = np.floor(h6).astype(np.int64) % 6
    f = h6 - np.floor(h6)
    p = v * (1 - s)
    q = v * (1 - s * f)
    t = v * (1 - s * (1 - f))
    r = np.choose(i, [v, q, p, p, t, v])
    g = np.choose(i, [t, v, v, q, p, p])
    b = np.choose(i, [p, p, t, v, v, q])
    return np.stack([r, g, b])


def hue_bin(h, bins):
    """Bin of each hue, computed in double: floor(h * bins), clamped to the last bin."""
    return np.minimum(np.floor(np.asarray(h, np.float64) * bins).astype(np.int64), bins - 1)


def hue_histogram(h, bins):
    """Normalised histogram of the hues (mass 1)."""
    c = np.bincount(hue_bin(h, bins), minlength=bins).astype(np.float64)
    return c / c.sum()


def exact_counts(target, npix):
    """Integer counts summing to npix from a histogram of mass 1: floors plus the largest remainders
    (ties to the lower bin)."""
    t = np.maximum(np.asarray(target, np.float64), 0.0)   # negative entries count as empty
    x = t / t.sum() * npix
    c = np.floor(x).astype(np.int64)
    rem = x - c
    short = npix - int(c.sum())
    order = np.lexsort((np.arange(len(x)), -rem))   # largest remainder first, then lower bin
    c[order[:short]] += 1
    return c


def target_hues(counts, bins):
    """Sorted target hues of exact counts: rank q in bin b gets (b + (q - C_b + 1/2) / c_b) / bins."""
    C = np.concatenate([[0], np.cumsum(counts)])
    q = np.arange(int(C[-1]))
    b = np.searchsorted(C, q, side="right") - 1
    return (b + (q - C[b] + 0.5) / counts[b]) / bins


def circular_sq(x, y):
    """Squared distance on the circle of circumference 1 between hues x and y (elementwise)."""
    d = np.abs(x - y)
    d = np.minimum(d, 1.0 - d)
    return d * d


def shift_cost(x, y, s):
    """sum_r d(x_r, y_{(r - s) mod n})^2 with d the distance on the unit circle."""
    return float(np.sum(circular_sq(x, np.roll(y, s))))


def all_shift_costs(x, y):
    """shift_cost for every s in [0, n), evaluated in blocks of shifts."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    n = len(x)
    r = np.arange(n)
    out = np.empty(n)
    step = max(1, min(n, (1 << 22) // max(n, 1)))
    for s0 in range(0, n, step):
        s = np.arange(s0, min(n, s0 + step))
        out[s0:s0 + len(s)] = np.sum(circular_sq(x[None, :], y[(r[None, :] - s[:, None]) % n]), axis=1)
    return out


def best_shift(x, y):
    """The least-cost cyclic shift: the first minimiser of shift_cost over every s in [0, n) (ties go
    to the smaller shift)."""
    return int(np.argmin(all_shift_costs(x, y)))


def strict_order(h):
    """Pixel indices sorted by (hue quantised to 32 bits, index)."""
    q = np.minimum(np.floor(np.asarray(h, np.float32).astype(np.float64) * 4294967296.0), 4294967295.0)
    return np.lexsort((np.arange(len(q)), q.astype(np.uint64)))


def specify(h, bins, target):
    """Periodic exact histogram specification of the hues h to the histogram `target`."""
    h = np.asarray(h, np.float32)
    npix = len(h)
    order = strict_order(h)
    y = target_hues(exact_counts(target, npix), bins)
    x = h[order].astype(np.float64)
    s = best_shift(x, y)
    out = np.empty(npix)
    out[order] = np.roll(y, s)     # rank r receives target rank (r - s) mod npix
    return out


def frames(rgb0, hist_path, bins):
    """Images u_t of section 5: the source's hues specified to each histogram of the path, with the
    source's saturation and value."""
    h, s, v = rgb_to_hsv(rgb0)
    return [hsv_to_rgb(specify(h, bins, ht), s, v) for ht in hist_path]
