"""The seeded scene generator: deterministic, and its ground truth is the plane of the front surface."""
import numpy as np

import scenes


def test_deterministic():
    a = scenes.config_pairs("vga_polygons")[0]
    b = scenes.config_pairs("vga_polygons")[0]
    assert np.array_equal(a.left, b.left) and np.array_equal(a.right, b.right)


def test_ground_truth_warp_consistency():
    sc = scenes.polygon_scene(200, 120, 99, n_poly=6, dmax=32, sigma=0.0)
    L, R, gt, occ = scenes.render(sc)
    H, W = L.shape
    vv, uu = np.mgrid[0:H, 0:W]
    x = np.rint(uu - gt).astype(int)
    ok = (~occ) & (x >= 0) & (np.abs(uu - gt - x) < 0.05)
    # noise-free: a visible pixel's texture reappears at x = u - d (up to sub-pixel resampling)
    diff = np.abs(L[ok].astype(int) - R[vv[ok], x[ok]].astype(int))
    assert np.median(diff) <= 2


def test_integer_shift_exact():
    p = scenes.integer_shift_pair(50, 20, 4, texture="iid")
    assert np.array_equal(p.right[:, :46], p.left[:, 4:])
