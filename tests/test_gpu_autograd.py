"""The hand-written backward behind torch.autograd.Function (render.render):
a loss built in torch from the rendered planes, loss.backward(), and the
leaves' .grad against the FP64 oracle's reverse pass and against central
finite differences of the oracle's forward (adjoint of Eqs. 2, 5, 6, 7)."""
import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _util import check_gradients, normwise  # noqa: E402

KEYS = ("xyz", "scale", "quat", "opacity", "rgb", "sem", "exposure")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render
    return render


def leaves(m, ex):
    f = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device="cuda", requires_grad=True)
    return [f(m.xyz), f(m.scale), f(m.quat), f(m.opacity), f(m.rgb), f(m.sem), f(ex)]


def torch_loss(out, cams, C, tg, lambda_c=1.0, lambda_s=0.06):
    """Masked L1 (three channels summed) + masked cross entropy of the
    composited logits, both over |M| (Eqs. 8-9), written in torch on the
    planar output of the views."""
    nch = 3 + C + 1
    l1, ce, nm, off = 0.0, 0.0, 0, 0
    for v, c in enumerate(cams):
        P = c.width * c.height
        pl = out[off: off + nch * P].view(nch, P)
        off += nch * P
        mk = torch.as_tensor(tg.mask[v].reshape(-1).astype(bool), device="cuda")
        trgb = torch.as_tensor(tg.rgb[v].reshape(3, -1), device="cuda")
        lab = torch.as_tensor(tg.label[v].reshape(-1).astype(np.int64), device="cuda")
        l1 = l1 + (pl[:3, mk] - trgb[:, mk]).abs().sum()
        ce = ce + torch.nn.functional.cross_entropy(pl[3:3 + C, mk].T, lab[mk], reduction="sum")
        nm += int(mk.sum())
    return (lambda_c * l1 + lambda_s * ce) / max(nm, 1)


def per_pixel(planar, cams, C, pix):
    """Planar flat vector -> (n_pix, 3+C+1) at an oracle pixel list."""
    nch = 3 + C + 1
    res = np.zeros((pix.shape[0], nch))
    off = 0
    for v, c in enumerate(cams):
        P = c.width * c.height
        pl = planar[off: off + nch * P].reshape(nch, c.height, c.width)
        s = pix[:, 0] == v
        res[s] = pl[:, pix[s, 2], pix[s, 1]].T
        off += nch * P
    return res


def check_against_oracle(m, cams, ex, grads, gout_pix, pix):
    gref = oracle.backward(m, cams, ex, pix, gout_pix)
    report = check_gradients({k: g.detach().cpu().numpy() for k, g in zip(KEYS, grads)}, gref.as_dict())
    return gref, report


@pytest.mark.parametrize("multiview", [False, True])
def test_loss_backward_through_autograd_matches_oracle(R, multiview):
    m = scenes.tiny_map(C=8)
    cams = [scenes.tiny_camera()]
    ex = np.array([[0.07, -0.02]], np.float32)
    if multiview:
        cams.append(scenes.bev_camera((3.0, 3.2), 80, res_m=0.07, height_m=20.0, exposure_idx=1))
        ex = np.array([[0.07, -0.02], [-0.05, 0.01]], np.float32)
    tg = scenes.random_targets(cams, 8, seed=11)
    rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
    lv = leaves(m, ex)
    out, fr = R.render(rr, cams, *lv)
    out.retain_grad()
    loss = torch_loss(out, cams, 8, tg)
    loss.backward()
    torch.cuda.synchronize()
    pix = oracle.full_pixels(cams)
    # the upstream gradient autograd handed to the backward, per pixel
    gout = per_pixel(out.grad.cpu().numpy().astype(np.float64), cams, 8, pix)
    # it is the loss gradient of Eqs. 8-9 (the oracle's, at the oracle's output,
    # except where |c' - cbar| is within rounding of the L1 kink)
    ref = oracle.render(m, cams, ex, pix)
    rgb, lb, mk = oracle.gather_targets(tg, pix)
    L, gl = oracle.loss(ref.out, rgb, lb, mk, 8)
    assert abs(float(loss.item()) - L) < 1e-4 * max(1.0, abs(L))
    kink = (np.abs(np.abs(gout[:, :3]) - np.abs(gl[:, :3])) > 1e-9).any(1)
    assert kink.sum() <= 8, kink.sum()
    assert np.abs(gout[~kink] - gl[~kink]).max() <= 1e-5 * np.abs(gl).max()
    check_against_oracle(m, cams, ex, [t.grad for t in lv], gout, pix)


def test_autograd_gradients_match_finite_differences(R):
    """Central differences (eps = 1e-4) of the FP64 oracle forward, for the
    linear functional <g, out> with g the upstream gradient autograd passed,
    on a sample of parameters of every type; samples whose perturbation
    changes a composited list (a threshold or stop decision flips) are left
    out and counted."""
    m = scenes.tiny_map(C=4)
    cams = [scenes.tiny_camera()]
    ex = np.array([[0.03, 0.01]], np.float32)
    tg = scenes.random_targets(cams, 4, seed=12)
    rr = R.Renderer(4, record_capacity=1 << 16, pair_capacity=1 << 20)
    lv = leaves(m, ex)
    out, fr = R.render(rr, cams, *lv)
    out.retain_grad()
    torch_loss(out, cams, 4, tg).backward()
    torch.cuda.synchronize()
    # a crop keeps the oracle's forward cheap; the loss functional is restricted to it
    pix = oracle.crop_pixels(0, 120, 100, 48, 40)
    gall = per_pixel(out.grad.cpu().numpy().astype(np.float64), cams, 4, oracle.full_pixels(cams))
    sel = (oracle.full_pixels(cams)[:, 2] >= 100) & (oracle.full_pixels(cams)[:, 2] < 140) & \
          (oracle.full_pixels(cams)[:, 1] >= 120) & (oracle.full_pixels(cams)[:, 1] < 168)
    gcrop = gall[sel]
    base = oracle.render(m, cams, ex, pix)
    ok = base.amb == 0
    gcrop[~ok] = 0.0                                  # ambiguity-band pixels take no part
    # GPU gradient of <gcrop, out_crop>: a second backward on a fresh forward of the same map
    lv2 = leaves(m, ex)
    out2, fr2 = R.render(rr, cams, *lv2)
    gplan = np.zeros(out2.numel(), np.float32)
    nch = 3 + 4 + 1
    W, H = cams[0].width, cams[0].height
    pl = gplan.reshape(nch, H, W)
    pl[:, pix[:, 2], pix[:, 1]] = gcrop.T
    (out2 * torch.as_tensor(gplan, device="cuda")).sum().backward()
    torch.cuda.synchronize()
    touched = np.nonzero(np.abs(oracle.backward(m, cams, ex, pix[ok], gcrop[ok]).rgb).sum(1))[0]
    assert len(touched) > 30
    rng = np.random.default_rng(0)
    eps = 1e-4
    rows, flips = [], 0
    kinds = [("xyz", 3), ("scale", 2), ("quat", 4), ("opacity", 1), ("rgb", 3), ("sem", 4)]
    for s in range(96):
        name, width = kinds[s % len(kinds)]
        i = int(rng.choice(touched))
        kk = int(rng.integers(0, width))
        vals, flip = [], False
        for d in (eps, -eps):
            mp = m.copy()
            arr = getattr(mp, name).astype(np.float64)
            arr.reshape(m.n, -1)[i, kk] += d
            setattr(mp, name, arr)
            rp = oracle.render(mp, cams, ex, pix[ok])
            flip |= not np.array_equal(rp.sig, base.sig[ok])
            vals.append(float((rp.out * gcrop[ok]).sum()))
        if flip:
            flips += 1
            continue
        fd = (vals[0] - vals[1]) / (2 * eps)
        gpu = float(dict(zip(KEYS, lv2))[name].grad.cpu().numpy().reshape(m.n, -1)[i, kk])
        rows.append((name, fd, gpu))
    assert len(rows) >= 80, (len(rows), flips)
    fd = np.array([r[1] for r in rows]); gg = np.array([r[2] for r in rows])
    assert np.abs(fd - gg).max() <= 1e-3 * np.abs(fd).max(), (np.abs(fd - gg).max(), np.abs(fd).max())


def test_backward_after_the_frame_was_rendered_again_raises(R):
    m = scenes.tiny_map(C=2)
    cams = [scenes.tiny_camera()]
    ex = np.zeros((1, 2), np.float32)
    rr = R.Renderer(2, record_capacity=1 << 16, pair_capacity=1 << 20)
    lv = leaves(m, ex)
    out, fr = R.render(rr, cams, *lv)
    out2, _ = R.render(rr, cams, *lv, frame=fr)      # the same frame: its state now belongs to out2
    with pytest.raises(RuntimeError, match="rendered again"):
        out.sum().backward()
    out2.sum().backward()                             # the latest forward is fine
    torch.cuda.synchronize()
    assert torch.isfinite(lv[4].grad).all() and lv[4].grad.abs().sum() > 0


def test_autograd_on_a_side_stream(R):
    """Forward and backward enqueued on a non-blocking side stream give the
    same gradients as on the default stream."""
    m = scenes.tiny_map(C=3)
    cams = [scenes.tiny_camera()]
    ex = np.array([[0.02, 0.0]], np.float32)
    rr = R.Renderer(3, record_capacity=1 << 16, pair_capacity=1 << 20)
    lv = leaves(m, ex)
    out, fr = R.render(rr, cams, *lv)
    (out * out).sum().backward()
    torch.cuda.synchronize()
    ref = [t.grad.clone() for t in lv]
    s = torch.cuda.Stream()
    lv2 = leaves(m, ex)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        out2, fr2 = R.render(rr, cams, *lv2)
        (out2 * out2).sum().backward()
    s.synchronize()
    for a, b in zip(lv2, ref):
        assert normwise(a.grad.cpu().numpy(), b.cpu().numpy()) < 1e-5
