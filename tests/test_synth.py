"""The seeded input generators follow the stated recipe: shapes in the ABI layout, mass 1, positivity,
determinism per seed, the mixed batch's size ranges, and hue image pairs that share saturation and value."""
import numpy as np

from paper_1501_04840_gb300 import synth


def test_rgb_pair_recipe():
    f0, f1 = synth.rgb_pair(40, 24, 8, 3)
    assert f0.shape == f1.shape == (3, 24, 40) and f0.dtype == np.float32
    for f in (f0, f1):
        assert abs(float(f.astype(np.float64).sum()) - 1.0) < 1e-6
        assert f.min() > 0
    assert not np.array_equal(f0, f1)
    g0, g1 = synth.rgb_pair(40, 24, 8, 3)
    assert np.array_equal(f0, g0) and np.array_equal(f1, g1)
    # pair s draws f0 from seed 2s and f1 from seed 2s + 1
    assert np.array_equal(f1, synth.rgb_blobs(40, 24, 8, 7))


def test_hue_pair_recipe():
    h0, h1 = synth.hue_pair(360, 2)
    assert h0.shape == h1.shape == (360,)
    for h in (h0, h1):
        assert abs(float(h.astype(np.float64).sum()) - 1.0) < 1e-6 and h.min() > 0


def test_mixed_batch_ranges():
    rgb, hue = synth.mixed_batch(0)
    assert len(rgb) == 16 and len(hue) == 64
    assert all(d["n1"] in (64, 96, 128, 192, 256) and d["n2"] in (64, 96, 128, 192, 256) for d in rgb)
    assert all(16 <= d["P"] <= 48 for d in rgb)
    assert all(64 <= d["n"] <= 720 and 16 <= d["P"] <= 64 for d in hue)
    assert synth.mixed_batch(0) == (rgb, hue)


def test_hue_image_pair_shares_saturation_and_value():
    a, b = synth.hue_image_pair(48, 1)
    assert a.shape == b.shape == (3, 48, 48)
    assert a.min() >= 0 and a.max() <= 1 and b.min() >= 0 and b.max() <= 1
    np.testing.assert_allclose(a.max(axis=0), b.max(axis=0), atol=1e-6)    # value
    np.testing.assert_allclose(a.min(axis=0), b.min(axis=0), atol=1e-6)    # value (1 - saturation)
    assert not np.allclose(a, b)
