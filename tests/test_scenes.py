"""The seeded input generator shared by the oracle and the CUDA path (CPU).

Pinned to SplitMix64's published first outputs, to the properties each draw
promises, and to the scene contract: with the noise off, every pixel the
ground truth marks as matched, whose match x - d lies in the image and is not
hidden behind a nearer surface, shows the same intensity in the right image
at x - d.
"""
import numpy as np
import pytest

from paper_1807_06271_gb300 import scenes


def test_splitmix64_reference_outputs():
    # the first three outputs of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014)
    r = scenes.Rng(0)
    got = [int(v) for v in r.draw(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # the stream continues where it stopped
    r2 = scenes.Rng(0)
    assert [int(v) for v in np.concatenate([r2.draw(1), r2.draw(2)])] == got


def test_draws_stay_in_their_ranges():
    r = scenes.Rng(1807)
    u = r.uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    k = r.integers(3, 9, 100000)
    assert k.min() == 3 and k.max() == 9
    assert np.all(np.bincount(k)[3:] > 100000 / 7 * 0.9)
    g = r.normal(100000)  # Irwin-Hall: mean 0, variance 12 * (1/12) = 1
    assert abs(g.mean()) < 0.02 and abs(g.var() - 1.0) < 0.03
    assert g.min() >= -6.0 and g.max() <= 6.0


def test_same_seed_same_bytes_different_seed_different_bytes():
    a = scenes.boxes_scene(96, 40, 64, seed=11)
    b = scenes.boxes_scene(96, 40, 64, seed=11)
    c = scenes.boxes_scene(96, 40, 64, seed=12)
    assert np.array_equal(a.left, b.left) and np.array_equal(a.right, b.right) and np.array_equal(a.gt, b.gt)
    assert not np.array_equal(a.left, c.left)


@pytest.mark.parametrize("make", [
    lambda: scenes.boxes_scene(160, 60, 64, seed=3, n_boxes=4, dlo=4, dhi=50, sigma=0.0),
    lambda: scenes.ground_scene(200, 90, 128, seed=4, n_obstacles=3, dlo=20, dhi=100, texture="value",
                                sigma=0.0, occlusion=0.0),
], ids=["boxes", "ground"])
def test_matched_pixels_appear_at_x_minus_d_without_noise(make):
    s = make()
    H, W = s.left.shape
    assert s.left.dtype == np.uint8 and s.right.dtype == np.uint8 and s.left.shape == s.right.shape
    # pixels whose match x - d lies in the image; of those landing on the same
    # right pixel the nearest (largest d) is the one the right view shows
    y, x = np.nonzero(s.gt >= 0)
    d = s.gt[y, x].astype(np.int64)
    inside = x - d >= 0
    y, x, d = y[inside], x[inside], d[inside]
    nearest = np.full((H, W), -1, np.int64)
    np.maximum.at(nearest, (y, x - d), d)
    shown = nearest[y, x - d] == d
    assert np.array_equal(s.right[y[shown], (x - d)[shown]], s.left[y[shown], x[shown]])
    # most of the image is matched and shown
    assert shown.sum() > 0.5 * H * W


def test_workload_scenes_have_the_workload_shapes():
    for name, w in scenes.WORKLOADS.items():
        s = scenes.scene_for(w, scenes.workload_seed(0))
        assert s.left.shape == (w.H, w.W) and s.right.shape == (w.H, w.W), name
        assert s.gt.max() < w.D, name
