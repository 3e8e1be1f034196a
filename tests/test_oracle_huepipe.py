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


def test_shift_search_is_the_exhaustive_minimum_on_small_inputs():
    h = _hues(300, 5)
    bins = 20
    rng = np.random.default_rng(6)
    target = rng.random(bins)
    target /= target.sum()
    order = hp.strict_order(h)
    x = h[order].astype(np.float64)
    y = hp.target_hues(hp.exact_counts(target, len(h)), bins)
    costs = [hp.shift_cost(x, y, s) for s in range(len(h))]
    assert hp.best_shift(x, y) == int(np.argmin(costs))
