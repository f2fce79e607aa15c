"""Fused Adam step (rogs_adam_step) against the FP64 oracle, and a short
optimisation of a perturbed map towards targets rendered from the original."""
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


def test_adam_groups_match_oracle(R):
    rng = np.random.default_rng(0)
    m = scenes.tiny_map(C=5)
    rr = R.Renderer(5, record_capacity=1 << 12, pair_capacity=1 << 12)
    st = R.SurfelTensors.from_map(m)
    ex = torch.as_tensor(rng.normal(0, 0.1, (3, 2)).astype(np.float32), device="cuda")
    opt = R.Adam(rr, st, ex, scene_size=5.0, total_steps=10)
    ref = {"z": m.xyz[:, 2].astype(np.float64), "scale": m.scale.ravel().astype(np.float64),
           "quat": m.quat.ravel().astype(np.float64), "opacity": m.opacity.astype(np.float64),
           "rgb": m.rgb.ravel().astype(np.float64), "sem": m.sem.ravel().astype(np.float64),
           "exposure": ex.cpu().numpy().ravel().astype(np.float64)}
    mom = {k: (np.zeros_like(v), np.zeros_like(v)) for k, v in ref.items()}
    xy0 = st.xyz[:, :2].clone()
    for t in range(1, 4):
        grads = R.zero_grads(st, ex)
        gnp = {}
        for k, g in grads.items():
            gv = rng.normal(0, 1e-2, tuple(g.shape)).astype(np.float32)
            g.copy_(torch.as_tensor(gv))
            gnp[k] = gv
        zl = oracle.z_learning_rate(t - 1, 10, 5.0)   # the schedule runs inside rogs_adam_step
        opt.step(grads)
        torch.cuda.synchronize()
        gmap = {"z": gnp["xyz"][:, 2], "scale": gnp["scale"].ravel(), "quat": gnp["quat"].ravel(),
                "opacity": gnp["opacity"], "rgb": gnp["rgb"].ravel(), "sem": gnp["sem"].ravel(),
                "exposure": gnp["exposure"].ravel()}
        for k in ref:
            lr = zl if k == "z" else R.PAPER_LR[k]
            ref[k], m1, v1 = oracle.adam_step(ref[k], gmap[k].astype(np.float64), *mom[k], lr=lr, t=t)
            mom[k] = (m1, v1)
        for g in grads.values():   # zeroed after use
            assert not g.any()
    got = {"z": st.xyz[:, 2], "scale": st.scale.ravel(), "quat": st.quat.ravel(), "opacity": st.opacity,
           "rgb": st.rgb.ravel(), "sem": st.sem.ravel(), "exposure": ex.ravel()}
    for k, v in got.items():
        a = v.cpu().numpy().astype(np.float64)
        lr = R.PAPER_LR.get(k, 5.0 * 1.6e-4)
        assert np.abs(a - ref[k]).max() <= 1e-6 * max(1.0, np.abs(ref[k]).max()) + 1e-4 * lr, k
    assert torch.equal(st.xyz[:, :2], xy0)          # x, y are not learnt


def test_z_rate_schedule_and_xy_clearing(R):
    """The z column's rate follows the log-linear decay inside the library and
    stays at its end value after decay_steps; the x and y gradients are cleared
    with the z gradient (x, y are not learnt), other columns are untouched."""
    from paper_2405_14342_gb300 import rogs
    rr = R.Renderer(2, record_capacity=1 << 12, pair_capacity=1 << 12)
    n = 1000
    xyz = torch.zeros(n, 3, device="cuda")
    g = torch.zeros(n, 3, device="cuda")
    mm, vv = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    lr0, lr1, D = 0.5, 0.005, 4
    for t in range(1, 8):
        g.fill_(1.0)
        z_before = xyz[:, 2].clone()
        rogs.rogs_adam_step(rr.ctx, [(xyz[:, 2], g[:, 2], mm, vv, n, 3, lr0, lr1, D, 2)], t)
        torch.cuda.synchronize()
        # with a constant gradient of 1 the bias-corrected Adam update is lr_t / (1 + eps)
        step = (z_before - xyz[:, 2]).cpu().numpy().astype(np.float64)
        lr_t = oracle.z_learning_rate(t - 1, D, 1.0, start=lr0, end=lr1)
        assert np.abs(step - lr_t).max() < 1e-5 * lr_t + 1e-7, (t, step[:3], lr_t)
        assert not g.any()
        assert not xyz[:, :2].any()
    with pytest.raises(rogs.RogsError):   # zero_lead must stay inside the stride
        rogs.rogs_adam_step(rr.ctx, [(xyz[:, 2], g[:, 2], mm, vv, n, 3, lr0, lr1, D, 3)], 1)
    with pytest.raises(rogs.RogsError):   # a decay needs positive ends
        rogs.rogs_adam_step(rr.ctx, [(xyz[:, 2], g[:, 2], mm, vv, n, 3, lr0, 0.0, D, 0)], 1)


def test_adam_rejects_bad_arguments(R):
    from paper_2405_14342_gb300 import rogs
    rr = R.Renderer(2, record_capacity=1 << 12, pair_capacity=1 << 12)
    p = torch.zeros(4, device="cuda")
    grp = [(p, p.clone(), p.clone(), p.clone(), 4, 1, 0.1)]
    with pytest.raises(rogs.RogsError) as ei:
        rogs.rogs_adam_step(rr.ctx, grp, 0)
    assert ei.value.status == rogs.ROGS_ERR_INVALID
    with pytest.raises(rogs.RogsError):
        rogs.rogs_adam_step(rr.ctx, grp * 17, 1)
    with pytest.raises(rogs.RogsError):
        rogs.rogs_adam_step(rr.ctx, [(p, p, p, p, 4, 0, 0.1)], 1)


def test_optimisation_reduces_the_loss(R):
    """Targets rendered from the tiny map; a colour- and height-perturbed copy
    is optimised with train_step + Adam; the loss falls."""
    m = scenes.tiny_map(C=8)
    gi = scenes.grid_index(m)
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 96, res_m=0.06, height_m=20.0)]
    ex = torch.zeros(1, 2, device="cuda")
    rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
    st0 = R.SurfelTensors.from_map(m)
    fr0 = rr.frame(cams)
    rr.forward(st0, fr0, ex)
    torch.cuda.synchronize()
    planes = [fr0.view(v, 8) for v in range(len(cams))]
    trgb = torch.cat([p[:3].reshape(3, -1) for p in planes], 1).contiguous()
    trgb = torch.cat([p[:3].reshape(-1) for p in planes]).contiguous()
    lab = torch.cat([p[3:11].argmax(0).to(torch.int32).reshape(-1) for p in planes]).contiguous()
    msk = torch.ones(lab.numel(), dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(4)
    m2 = m.copy()
    m2.rgb = np.clip(m2.rgb + rng.normal(0, 0.2, m2.rgb.shape), 0, 1).astype(np.float32)
    st = R.SurfelTensors.from_map(m2, grid_index=gi)
    opt = R.Adam(rr, st, ex, scene_size=6.4, total_steps=30, lr=dict(R.PAPER_LR, rgb=0.02))
    grads = R.zero_grads(st, ex)
    fr = rr.frame(cams)
    loss = torch.empty(1, device="cuda")
    losses = []
    for t in range(30):
        rr.train_step(st, fr, ex, trgb, lab, msk, loss, grads, lambda_smooth=0.003)
        losses.append(float(loss.item()))
        opt.step(grads)
    torch.cuda.synchronize()
    assert losses[-1] < 0.7 * losses[0], losses
