"""Pins of the hue image pipeline reference (oracle/huepipe.py): HSV against
Python's colorsys, exactness of the histogram specification, its behaviour on
targets that are the source itself or the source rotated, and the shift
search against the exhaustive minimum."""
import colorsys

import numpy as np
import pytest

from oracle import huepipe as hp


def _pixels(n, seed):
    rng = np.random.default_rng(seed)
    rgb = rng.random((3, n))
    rgb[:, :10] = [[0, 1, 0, 0, 1, 1, 0.5, 0.2, 1, 0], [0, 0, 1, 0, 1, 0, 0.5, 0.2, 1, 1],
                   [0, 0, 0, 1, 0, 1, 0.5, 0.2, 1, 1]]   # black, pure colours, greys, white, cyan
    return rgb


def test_hsv_against_colorsys():
    rgb = _pixels(2000, 0)
    h, s, v = hp.rgb_to_hsv(rgb)
    ref = np.array([colorsys.rgb_to_hsv(*rgb[:, i]) for i in range(rgb.shape[1])]).T
    np.testing.assert_allclose(h, ref[0], atol=1e-12)
    np.testing.assert_allclose(s, ref[1], atol=1e-12)
    np.testing.assert_allclose(v, ref[2], atol=1e-12)
    back = hp.hsv_to_rgb(h, s, v)
    ref_back = np.array([colorsys.hsv_to_rgb(h[i], s[i], v[i]) for i in range(len(h))]).T
    np.testing.assert_allclose(back, ref_back, atol=1e-12)
    np.testing.assert_allclose(back, rgb, atol=1e-12)


def _hues(n, seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([(0.15 + 0.05 * rng.standard_normal(n // 2)) % 1.0,
                           (0.95 + 0.08 * rng.standard_normal(n - n // 2)) % 1.0]).astype(np.float32)


def test_specification_is_exact():
    h = _hues(5000, 1)
    bins = 36
    rng = np.random.default_rng(2)
    target = rng.random(bins) ** 3
    target /= target.sum()
    out = hp.specify(h, bins, target)
    counts = np.bincount(hp.hue_bin(out, bins), minlength=bins)
    assert np.array_equal(counts, hp.exact_counts(target, len(h)))
    assert np.all((out >= 0) & (out < 1))


def test_specification_to_the_source_histogram_keeps_every_bin():
    h = _hues(3000, 3)
    bins = 60
    out = hp.specify(h, bins, hp.hue_histogram(h, bins))
    assert np.array_equal(hp.hue_bin(out, bins), hp.hue_bin(h, bins))


@pytest.mark.parametrize("k", [1, 3, 58, 59])
def test_specification_to_a_slightly_rotated_histogram_rotates_every_pixel(k):
    """A target that is the source histogram turned by up to three bins, either way (58, 59 turn back
    across the 0 = 1 seam): the least-cost cut moves every pixel by exactly that rotation.  (For larger
    turns of this two-mode source the least-cost cyclic assignment is no longer the rotation: the
    targets are spread evenly inside their bins, and moving a few pixels across to the other mode
    becomes cheaper.)"""
    h = _hues(3000, 4)
    bins = 60
    out = hp.specify(h, bins, np.roll(hp.hue_histogram(h, bins), k))
    assert np.array_equal(hp.hue_bin(out, bins), (hp.hue_bin(h, bins) + k) % bins)


def test_exact_counts_by_hand():
    """Largest remainders, worked by hand: shares 3.5, 2.1, 1.4 of 7 pixels floor to 3, 2, 1 and the one
    pixel left goes to the largest remainder (bin 0); equal remainders go to the lower bin; negative
    entries count as empty and the rest is renormalised."""
    assert hp.exact_counts([0.5, 0.3, 0.2], 7).tolist() == [4, 2, 1]
    assert hp.exact_counts([1 / 3, 1 / 3, 1 / 3], 4).tolist() == [2, 1, 1]
    assert hp.exact_counts([0.5, -0.1, 0.6], 11).tolist() == [5, 0, 6]
    assert hp.exact_counts([0.1, 0.2, 0.3, 0.4], 10).tolist() == [1, 2, 3, 4]


def test_target_hues_by_hand():
    """Counts (2, 0, 1) over 3 bins: the two ranks of bin 0 sit at its quarter points, the one rank of
    bin 2 at its centre."""
    np.testing.assert_allclose(hp.target_hues(np.array([2, 0, 1]), 3), [0.25 / 3, 0.75 / 3, 2.5 / 3], rtol=0,
                               atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_best_cyclic_shift_is_the_optimal_assignment(seed):
    """For sorted points on the circle with a cost convex in the circular distance, an optimal matching
    of two equal-size sets is a cyclic shift of the sorted orders.  The Hungarian method (scipy's
    linear_sum_assignment) over all permutations pins the shift search: the least-cost cyclic shift
    reaches the optimal assignment cost."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(40, 160))
    x = np.sort(_hues(n, seed).astype(np.float64))
    y = np.sort((rng.normal(rng.random(), 0.05 + 0.3 * rng.random(), n)) % 1.0)
    d = np.abs(x[:, None] - y[None, :])
    d = np.minimum(d, 1.0 - d)
    r, c = linear_sum_assignment(d * d)
    optimal = float(np.sum((d * d)[r, c]))
    s = hp.best_shift(x, y)
    assert hp.shift_cost(x, y, s) <= optimal * (1 + 1e-12) + 1e-15


def _bump_counts(n, bins, centre=0.97, width=0.03, support=0.1):
    """Exact counts of a truncated Gaussian bump on the circle (support 0.2 of the circle, across the
    0 = 1 seam for the default centre)."""
    c = (np.arange(bins) + 0.5) / bins
    d = np.abs(c - centre)
    d = np.minimum(d, 1.0 - d)
    dens = np.where(d < support, np.exp(-0.5 * (d / width) ** 2), 0.0)
    return hp.exact_counts(dens / dens.sum(), n)


@pytest.mark.parametrize("n,k", [(4096, 1), (4096, 5), (4096, -3), (8192, 2)])
def test_rotated_bump_is_cut_at_the_rotation(n, k):
    """A closed-form case on thousands of pixels: the source hues sit at the target hues of their own
    exact counts, and the target is that histogram turned by k bins.  Every target hue is then a source
    hue moved by delta = k / bins, and with all mass inside an arc shorter than half the circle the
    rotation is the optimal transport (on an arc, translation is the monotone and hence optimal map):
    cost n delta^2.  The sorted target is the sorted source rotated by the m pixels that cross the seam,
    so the least-cost shift is -m mod n when they wrap forwards (k > 0) and m when backwards (k < 0)."""
    bins = 90
    counts = _bump_counts(n, bins)
    x = hp.target_hues(counts, bins)
    y = hp.target_hues(np.roll(counts, k), bins)
    delta = k / bins
    if k > 0:
        expect = (n - int(np.sum(x + delta >= 1.0))) % n
    else:
        expect = int(np.sum(x + delta < 0.0))
    s = hp.best_shift(x, y)
    assert s == expect
    assert hp.shift_cost(x, y, s) == pytest.approx(n * delta ** 2, rel=1e-12)
