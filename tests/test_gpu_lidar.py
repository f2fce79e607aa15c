"""LiDAR elevation supervision (rogs_elev_targets, rogs_elev_loss) against
the FP64 oracle: nearest points by brute force, L_z and its gradient."""
import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render
    return render


def _check_targets(xy, pts, radius, got):
    """Count surfels whose target is not the z of a point at the minimal
    distance (ties within FP32 rounding allowed) or that are NaN although a
    point lies clearly within the radius."""
    ref, idx = oracle.nearest_elevation(xy, pts, radius)
    P = pts.astype(np.float64)
    bad = 0
    for i in np.nonzero(~(np.isnan(got) & np.isnan(ref)) & ~(got == ref))[0]:
        d2 = ((P[:, :2] - xy[i]) ** 2).sum(1)
        dmin = d2.min()
        tol = 1e-5 * max(radius * radius, dmin) + 1e-9
        if np.isnan(got[i]):      # dropped: the nearest point must sit on the radius
            ok = abs(dmin - radius * radius) <= tol
        else:
            near = d2 <= dmin + tol
            ok = bool(np.any(P[near, 2].astype(np.float32) == got[i])) and (dmin <= radius * radius + tol)
        bad += not ok
    return bad


def test_targets_match_brute_force(R):
    m = scenes.tiny_map(C=2)
    pts = scenes.lidar_points(lambda x, y: 0.02 * np.sin(x) * np.cos(y), (-0.2, 6.5), (-0.2, 6.5), 20000, seed=3)
    pts[:50] = pts[50:100]                        # duplicate points: equal distances
    rr = R.Renderer(2, record_capacity=1 << 12, pair_capacity=1 << 12)
    st = R.SurfelTensors.from_map(m)
    dp = torch.as_tensor(pts, device="cuda")
    for radius in (0.05, 0.1, 0.3):
        zt = rr.elev_targets(st, dp, radius).cpu().numpy()
        assert _check_targets(m.xyz[:, :2].astype(np.float64), pts, radius, zt) == 0
    zt = rr.elev_targets(st, dp[:0], 0.1).cpu().numpy()    # an empty cloud: no targets
    assert np.isnan(zt).all()


def test_loss_and_gradient_match_oracle(R):
    m = scenes.tiny_map(C=2)
    pts = scenes.lidar_points(lambda x, y: 0.02 * np.sin(x) * np.cos(y), (0.0, 6.3), (0.0, 4.0), 8000, seed=4)
    rr = R.Renderer(2, record_capacity=1 << 12, pair_capacity=1 << 12)
    st = R.SurfelTensors.from_map(m)
    zt = rr.elev_targets(st, torch.as_tensor(pts, device="cuda"), 0.1)
    lam = 0.02
    loss = torch.full((1,), 0.5, device="cuda")     # the loss is added to what is there
    g = torch.zeros_like(st.xyz)
    rr.elev_loss(st, zt, lam, loss, g)
    torch.cuda.synchronize()
    ztn = zt.cpu().numpy().astype(np.float64)
    L, gr = oracle.elev_loss(m.xyz[:, 2].astype(np.float64), ztn)
    assert abs(loss.item() - (0.5 + lam * L)) <= 1e-5 * (0.5 + lam * L)
    gz = g[:, 2].cpu().numpy()
    assert np.abs(gz - lam * gr).max() <= 1e-5 * lam * max(np.abs(gr).max(), 1e-12)
    assert not g[:, :2].any()
    assert np.isnan(ztn).any() and np.isfinite(ztn).any()    # both cases exercised


def test_strip_scale_targets(R):
    m, field = scenes.strip_map(C=2, seed=0)
    h = lambda x, y: field(x, y)[0]
    pts = scenes.lidar_points(h, (0.0, 400.0), (0.0, 40.0), 2_000_000, seed=6)
    rr = R.Renderer(2, record_capacity=1 << 12, pair_capacity=1 << 12)
    st = R.SurfelTensors.from_map(m)
    zt = rr.elev_targets(st, torch.as_tensor(pts, device="cuda"), 0.1).cpu().numpy()
    rng = np.random.default_rng(7)
    sel = rng.choice(m.n, 2000, replace=False)
    # the brute force only needs the points near the sampled surfels
    order = np.argsort(pts[:, 0], kind="stable")
    xs = pts[order, 0]
    near = []
    for x, y in m.xyz[sel, :2]:
        a, b = np.searchsorted(xs, [x - 0.2, x + 0.2])
        cand = order[a:b]
        near.append(cand[np.abs(pts[cand, 1] - y) < 0.2])
    sub = pts[np.unique(np.concatenate(near))]
    assert _check_targets(m.xyz[sel, :2].astype(np.float64), sub, 0.1, zt[sel]) == 0
