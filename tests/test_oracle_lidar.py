"""Pins of the FP64 LiDAR elevation-loss oracle (RoGs Sec. 3.3.2, L_z), CPU only."""
import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes


def test_single_point_and_radius():
    xy = np.array([[0.0, 0.0], [0.3, 0.0], [1.0, 1.0], [0.7, 0.0]])
    pts = np.array([[0.1, 0.0, 2.5]])
    zb, idx = oracle.nearest_elevation(xy, pts, radius=0.5)
    np.testing.assert_array_equal(zb[:2], [2.5, 2.5])
    assert np.isnan(zb[2]) and idx[2] == -1
    assert np.isnan(zb[3]) and idx[3] == -1      # 0.6 m away: outside 0.5 m (though 0.6^2 < 0.5)
    # a radius above 1 m: 1.5 m away is inside 2 m (though 1.5^2 > 2)
    zb2, idx2 = oracle.nearest_elevation(np.array([[1.6, 0.0]]), pts, radius=2.0)
    assert zb2[0] == 2.5 and idx2[0] == 0


def test_points_on_the_surfels_pick_their_own():
    x, y = scenes.grid_xy(20, 10, spacing=0.1)
    xy = np.stack([x, y], -1)
    rng = np.random.default_rng(0)
    z = rng.normal(size=x.size)
    pts = np.stack([x, y, z], -1)[rng.permutation(x.size)]
    zb, idx = oracle.nearest_elevation(xy, pts, radius=0.04)
    np.testing.assert_array_equal(zb, z)


def test_matches_a_kd_tree_and_ties_take_the_lowest_index():
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 10, (3000, 3))
    xy = rng.uniform(0, 10, (500, 2))
    zb, idx = oracle.nearest_elevation(xy, pts, radius=100.0)
    d, j = spatial.cKDTree(pts[:, :2]).query(xy)
    np.testing.assert_array_equal(idx, j)
    # two points at the same distance: the lower index wins
    pts2 = np.array([[1.0, 0.0, 5.0], [-1.0, 0.0, 7.0]])
    zb2, idx2 = oracle.nearest_elevation(np.zeros((1, 2)), pts2, radius=2.0)
    assert idx2[0] == 0 and zb2[0] == 5.0


def test_loss_closed_form_and_finite_differences():
    z = np.array([1.0, 2.0, -0.5, 0.25])
    zb = np.array([0.5, np.nan, 0.0, 0.25])
    L, g = oracle.elev_loss(z, zb)
    assert L == pytest.approx(0.25 + 0.25)
    np.testing.assert_allclose(g, [1.0, 0.0, -1.0, 0.0])
    eps = 1e-6
    for i in range(4):
        zp, zm = z.copy(), z.copy()
        zp[i] += eps
        zm[i] -= eps
        fd = (oracle.elev_loss(zp, zb)[0] - oracle.elev_loss(zm, zb)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-6
