"""FP64 oracle of the LiDAR elevation loss (test infrastructure only).

RoGs Sec. 3.3.2 (LiDAR supervision): L_z = sum_i (z_i - zbar_i)^2, where
zbar_i is the elevation of the point of the LiDAR cloud nearest to surfel i
in the xy-plane.  Readings (not stated in the paper): only points within a
radius r of the surfel in xy are considered (the paper's elevation metric
queries within 0.1 m); a surfel with none takes no L_z term; among points at
the same distance the one with the lowest index is taken.
"""
from __future__ import annotations

import numpy as np


def nearest_elevation(surfel_xy, points, radius, chunk=2048):
    """zbar [n] (NaN where no point lies within `radius`) and the chosen point
    index [n] (-1 where none), by brute force over all points."""
    sxy = np.asarray(surfel_xy, np.float64)
    P = np.asarray(points, np.float64)
    n = sxy.shape[0]
    zbar = np.full(n, np.nan)
    idx = np.full(n, -1, np.int64)
    if P.shape[0] == 0:
        return zbar, idx
    for a in range(0, n, chunk):
        d2 = ((sxy[a:a + chunk, None, :] - P[None, :, :2]) ** 2).sum(-1)
        j = np.argmin(d2, axis=1)                       # first minimum = lowest index
        dmin = d2[np.arange(j.size), j]
        ok = dmin <= radius * radius
        zbar[a:a + chunk][ok] = P[j[ok], 2]
        idx[a:a + chunk][ok] = j[ok]
    return zbar, idx


def elev_loss(z, zbar):
    """(L_z, dL/dz) over the surfels with a target (finite zbar)."""
    z = np.asarray(z, np.float64)
    zbar = np.asarray(zbar, np.float64)
    has = np.isfinite(zbar)
    d = np.where(has, z - np.where(has, zbar, 0.0), 0.0)
    return float(np.sum(d * d)), 2.0 * d
