"""FP64 oracle of the elevation smoothness loss (test infrastructure only).

RoGs Sec. 3.3.2 (the smoothness equation): L_smooth = (1/K) sum_i sum_{j in N(i)}
(z_i - z_j)^2 with K = 4 neighbours, and supplementary "Smooth Loss K Nearest
Neighbor Acceleration": the neighbours are looked up through the grid index
map (vertex -> surfel id, -1 off the road) as the surfels at the vertices
above, below, left and right; a neighbour vertex that is off the grid or
off the road is replaced by the surfel itself.

The gradient is the literal adjoint of that sum: every ordered pair (i, j)
adds 2 (z_i - z_j) / K to dL/dz_i and subtracts it from dL/dz_j.  It does not
use the symmetry of the neighbour relation.
"""
from __future__ import annotations

import numpy as np

# (row, column) offsets of the four neighbours: up, down, left, right
NEIGHBOURS = ((-1, 0), (1, 0), (0, -1), (0, 1))


def neighbour_ids(grid_index: np.ndarray) -> np.ndarray:
    """(n, 4) surfel ids of each surfel's four neighbours (self where the
    neighbour vertex is off the grid or holds no surfel)."""
    gi = np.asarray(grid_index, dtype=np.int64)
    H, W = gi.shape
    n = int(gi.max()) + 1 if (gi >= 0).any() else 0
    out = np.zeros((n, 4), np.int64)
    rows, cols = np.nonzero(gi >= 0)
    ids = gi[rows, cols]
    for k, (dr, dc) in enumerate(NEIGHBOURS):
        rr, cc = rows + dr, cols + dc
        inside = (rr >= 0) & (rr < H) & (cc >= 0) & (cc < W)
        nb = np.where(inside, gi[np.clip(rr, 0, H - 1), np.clip(cc, 0, W - 1)], -1)
        out[ids, k] = np.where(nb >= 0, nb, ids)
    return out


def smooth_loss(z: np.ndarray, grid_index: np.ndarray, K: int = 4):
    """(L_smooth, dL/dz) in FP64 for surfel heights z [n]."""
    z = np.asarray(z, dtype=np.float64)
    nb = neighbour_ids(grid_index)
    n = nb.shape[0]
    i = np.repeat(np.arange(n), 4)
    j = nb.ravel()
    d = z[i] - z[j]
    L = float(np.sum(d * d)) / K
    g = np.zeros(z.shape[0])
    np.add.at(g, i, 2.0 * d / K)
    np.add.at(g, j, -2.0 * d / K)
    return L, g
