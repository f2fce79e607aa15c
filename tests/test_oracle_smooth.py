"""Pins of the FP64 smoothness-loss oracle (RoGs Sec. 3.3.2 smoothness loss,
supplementary "Smooth Loss K Nearest Neighbor Acceleration"), CPU only."""
import numpy as np

import oracle
from paper_2405_14342_gb300 import scenes


def _plane_grid(H, W, a, b, h=0.1):
    x, y = scenes.grid_xy(W, H, spacing=h)
    z = a * x + b * y
    gi = np.arange(H * W, dtype=np.int32).reshape(H, W)
    return z, gi


def test_plane_closed_form():
    """z = a x + b y on a full H x W grid: every horizontal ordered pair adds
    (a h)^2, every vertical one (b h)^2, edge neighbours are self (0)."""
    H, W, a, b, h = 7, 11, 0.3, -0.7, 0.1
    z, gi = _plane_grid(H, W, a, b, h)
    L, g = oracle.smooth_loss(z, gi)
    expect = (2 * H * (W - 1) * (a * h) ** 2 + 2 * (H - 1) * W * (b * h) ** 2) / 4.0
    assert abs(L - expect) < 1e-12 * max(1.0, expect)
    # interior columns cancel; the left column lacks its left neighbour, the right one its right
    G = g.reshape(H, W)
    np.testing.assert_allclose(G[1:-1, 1:-1], 0.0, atol=1e-12)
    np.testing.assert_allclose(G[1:-1, 0], -a * h, atol=1e-12)
    np.testing.assert_allclose(G[1:-1, -1], a * h, atol=1e-12)
    np.testing.assert_allclose(G[0, 1:-1], -b * h, atol=1e-12)
    np.testing.assert_allclose(G[-1, 1:-1], b * h, atol=1e-12)


def test_interior_neighbours_are_the_four_nearest():
    """Away from the border the grid lookup returns exactly the 4 nearest
    surfels in xy (brute force over all pairs)."""
    H, W = 9, 8
    x, y = scenes.grid_xy(W, H, spacing=0.1)
    gi = np.arange(H * W, dtype=np.int32).reshape(H, W)
    nb = oracle.neighbour_ids(gi)
    xy = np.stack([x, y], -1)
    for r in range(1, H - 1):
        for c in range(1, W - 1):
            i = gi[r, c]
            d = np.linalg.norm(xy - xy[i], axis=1)
            d[i] = np.inf
            near = set(np.argsort(d, kind="stable")[:4].tolist())
            assert set(nb[i].tolist()) == near
            assert np.sort(d)[4] > np.sort(d)[3] + 1e-9   # the four are unambiguous


def test_unordered_pair_form_and_shift_invariance():
    """L = 1/2 sum over unordered adjacent on-road pairs of (z_i - z_j)^2;
    adding a constant changes neither L nor the gradient, whose sum is 0."""
    m = scenes.tiny_map(C=2)
    m2, gi = scenes.with_holes(m, frac=0.3, seed=3)
    rng = np.random.default_rng(0)
    z = m2.xyz[:, 2].astype(np.float64) + rng.normal(0, 0.01, m2.n)
    L, g = oracle.smooth_loss(z, gi)
    H, W = gi.shape
    acc = 0.0
    for r in range(H):
        for c in range(W):
            i = gi[r, c]
            if i < 0:
                continue
            if c + 1 < W and gi[r, c + 1] >= 0:
                acc += (z[i] - z[gi[r, c + 1]]) ** 2
            if r + 1 < H and gi[r + 1, c] >= 0:
                acc += (z[i] - z[gi[r + 1, c]]) ** 2
    assert abs(L - 0.5 * acc) < 1e-12 * max(1.0, acc)
    L2, g2 = oracle.smooth_loss(z + 3.7, gi)
    assert abs(L2 - L) < 1e-9 * max(1.0, L)
    np.testing.assert_allclose(g2, g, atol=1e-9)
    assert abs(g.sum()) < 1e-9


def test_isolated_surfel_and_finite_differences():
    gi = np.array([[0, -1, 1], [-1, -1, 2], [3, 4, -1]], np.int32)
    z = np.array([0.5, -0.2, 0.1, 0.3, 0.9])
    L, g = oracle.smooth_loss(z, gi)
    assert g[0] == 0.0                       # surfel 0 has no on-road neighbour
    eps = 1e-6
    for i in range(z.size):
        zp, zm = z.copy(), z.copy()
        zp[i] += eps
        zm[i] -= eps
        fd = (oracle.smooth_loss(zp, gi)[0] - oracle.smooth_loss(zm, gi)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-8
    # only pairs (1,2) vertical and (3,4) horizontal: L = ((0.1+0.2)^2 + (0.9-0.3)^2) / 2
    assert abs(L - ((0.3) ** 2 + 0.6 ** 2) / 2.0) < 1e-12
