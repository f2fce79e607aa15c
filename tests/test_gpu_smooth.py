"""Elevation smoothness loss (rogs_smooth_loss) against the FP64 oracle:
tiny maps with off-road holes, the 1.6M-surfel strip, degenerate grids."""
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


def _run(R, m, gi, lam=0.003, grad=True):
    rr = R.Renderer(m.num_classes, record_capacity=1 << 12, pair_capacity=1 << 12)
    st = R.SurfelTensors.from_map(m, grid_index=gi)
    g = torch.zeros_like(st.xyz) if grad else None
    loss = rr.smooth_loss(st, lam, grad_xyz=g)
    torch.cuda.synchronize()
    return float(loss.item()), (g.cpu().numpy() if grad else None), rr, st


def test_tiny_with_holes_matches_oracle(R):
    m = scenes.tiny_map(C=2)
    m2, gi = scenes.with_holes(m, frac=0.3, seed=3)
    rng = np.random.default_rng(1)
    m2.xyz[:, 2] += rng.normal(0, 0.02, m2.n).astype(np.float32)
    lam = 0.003
    L, g, _, _ = _run(R, m2, gi, lam)
    Lr, gr = oracle.smooth_loss(m2.xyz[:, 2].astype(np.float64), gi)
    assert abs(L - lam * Lr) <= 1e-5 * lam * Lr
    gz = g[:, 2].astype(np.float64)
    assert np.abs(gz - lam * gr).max() <= 1e-5 * lam * np.abs(gr).max()
    assert not g[:, :2].any()                      # only dz is touched


def test_strip_scale_matches_oracle(R):
    m, _ = scenes.strip_map(C=2, seed=0)
    gi = scenes.grid_index(m)
    lam = 1.0
    L, g, rr, st = _run(R, m, gi, lam)
    Lr, gr = oracle.smooth_loss(m.xyz[:, 2].astype(np.float64), gi)
    assert abs(L - Lr) <= 1e-5 * Lr
    gz = g[:, 2].astype(np.float64)
    assert np.abs(gz - gr).max() <= 1e-5 * np.abs(gr).max()
    # fixed summation order: bit-identical loss on a second call
    L2 = float(rr.smooth_loss(st, lam).item())
    assert L2 == L


def test_gradient_accumulates_and_degenerate_grids(R):
    m = scenes.tiny_map(C=2)
    gi = scenes.grid_index(m)
    rr = R.Renderer(2, record_capacity=1 << 12, pair_capacity=1 << 12)
    st = R.SurfelTensors.from_map(m, grid_index=gi)
    g = torch.zeros_like(st.xyz)
    rr.smooth_loss(st, 0.5, grad_xyz=g)
    g1 = g.clone()
    rr.smooth_loss(st, 0.5, grad_xyz=g)
    torch.cuda.synchronize()
    assert torch.allclose(g, 2 * g1, rtol=1e-6, atol=0)
    # no on-road vertex: zero loss, no gradient
    empty = np.full((5, 7), -1, np.int32)
    st_e = R.SurfelTensors.from_map(m, grid_index=empty)
    g0 = torch.zeros_like(st.xyz)
    assert float(rr.smooth_loss(st_e, 1.0, grad_xyz=g0).item()) == 0.0
    assert not g0.any()
    # one row: only left/right neighbours
    row = np.arange(10, dtype=np.int32)[None, :]
    L, gr = oracle.smooth_loss(m.xyz[:10, 2].astype(np.float64), row)
    st_r = R.SurfelTensors.from_map(m, grid_index=row)
    assert abs(float(rr.smooth_loss(st_r, 1.0).item()) - L) <= 1e-5 * max(L, 1e-12)


def test_missing_grid_is_rejected(R):
    from paper_2405_14342_gb300 import rogs
    m = scenes.tiny_map(C=2)
    rr = R.Renderer(2, record_capacity=1 << 12, pair_capacity=1 << 12)
    st = R.SurfelTensors.from_map(m)
    with pytest.raises(rogs.RogsError) as ei:
        rr.smooth_loss(st, 1.0)
    assert ei.value.status == rogs.ROGS_ERR_INVALID


def test_training_step_adds_the_smoothness_term(R):
    """rogs_train_step with lambda_smooth: the loss gains lambda L_smooth and
    only the z column of the position gradient changes, by lambda dL/dz."""
    m = scenes.tiny_map(C=8)
    gi = scenes.grid_index(m)
    cams = [scenes.tiny_camera()]
    ex = torch.zeros(1, 2, device="cuda")
    rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
    st = R.SurfelTensors.from_map(m, grid_index=gi)
    trgb, lab, msk = R.targets_to_device(scenes.random_targets(cams, 8, seed=9))
    lam = 0.25
    res = []
    for ls in (0.0, lam):
        fr = rr.frame(cams)
        loss = torch.empty(1, device="cuda")
        grads = R.zero_grads(st, ex)
        rr.train_step(st, fr, ex, trgb, lab, msk, loss, grads, lambda_smooth=ls)
        torch.cuda.synchronize()
        res.append((loss.item(), {k: v.cpu().numpy() for k, v in grads.items()}))
    Lr, gr = oracle.smooth_loss(m.xyz[:, 2].astype(np.float64), gi)
    assert abs((res[1][0] - res[0][0]) - lam * Lr) <= 1e-5 * max(1.0, abs(res[1][0]))
    # the rendering gradients are atomic sums: equal up to FP32 summation order
    d = res[1][1]["xyz"].astype(np.float64) - res[0][1]["xyz"]
    ref = np.abs(res[0][1]["xyz"]).max()
    assert np.abs(d[:, :2]).max() <= 1e-6 * ref
    tol = 1e-5 * lam * np.abs(gr).max() + 1e-6 * ref
    assert np.abs(d[:, 2] - lam * gr).max() <= tol
    for k in res[0][1]:
        if k != "xyz":
            a0, a1 = res[0][1][k].astype(np.float64), res[1][1][k]
            assert np.abs(a1 - a0).max() <= 1e-6 * max(np.abs(a0).max(), 1e-30), k
