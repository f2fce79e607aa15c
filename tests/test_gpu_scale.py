"""CUDA path vs the FP64 oracle at the workloads' full sizes, on sampled
outputs, plus the equalities that must hold at any size:

* scene config (1.6M surfels, 6 x 960x540): sampled pixels (road half and a
  band of horizon rows, where tile lists are longest) at 1e-4; and the fused
  training step (loss + backward + grid smoothness, the bench's tile and sort
  chunk) with the loss mask on a pixel sample, every gradient tensor against
  the FP64 oracle (1e-3, normwise and element-wise: _util.check_gradients);
* batching config (48 views of uneven size in one call): every view equals
  the same view rendered alone, bit for bit, and sampled pixels match the
  oracle;
* graph-captured step == eager step;
* differentiation config (4.19M-surfel grid road network, 640x360): GPU
  gradients of a loss on the 64x64 crop vs the FP64 reverse pass (1e-3,
  normwise and element-wise) and vs central finite differences of the FP64
  forward (eps 1e-4) on 512 sampled parameters of every type, at 1e-3.
"""
import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _util import check_gradients, gpu_pixels, gpu_state_T, gpu_tile_lists, normwise, pixel_index, planar_grad_from_pixels  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render
    return render


@pytest.fixture(scope="module")
def strip():
    m, field = scenes.strip_map(C=19)
    return m, field


def sample_pixels(cams, n_per_view, seed, band=True):
    rng = np.random.default_rng(seed)
    out = []
    for v, c in enumerate(cams):
        u = rng.integers(0, c.width, n_per_view)
        y = rng.integers(c.height // 2, c.height, n_per_view)
        out.append(np.stack([np.full(n_per_view, v), u, y], -1))
        if band:   # rows just below the horizon: the 40 m end of the box, longest lists
            cy = int(c.cy)
            yy, uu = np.meshgrid(np.arange(cy + 8, cy + 40, 4), np.arange(c.width // 2 - 64, c.width // 2 + 64, 8),
                                 indexing="ij")
            out.append(np.stack([np.full(uu.size, v), uu.ravel(), yy.ravel()], -1))
    return np.ascontiguousarray(np.concatenate(out).astype(np.int32))


def check_pixels(fr, C, ref, pix, depth_scale=40.0, tol=1e-4):
    got = gpu_pixels(fr, C, pix)
    ok = ref.amb == 0
    assert (~ok).sum() <= max(4, 1e-3 * len(pix))
    assert np.abs(got[ok, :3] - ref.out[ok, :3]).max() < tol
    assert np.abs(got[ok, 3:3 + C] - ref.out[ok, 3:3 + C]).max() < tol
    assert (np.abs(got[ok, 3 + C] - ref.out[ok, 3 + C]) / depth_scale).max() < tol
    T = gpu_state_T(fr)[pixel_index(fr, pix)]
    assert np.abs(T[ok] - ref.T[ok]).max() < tol


def test_scene_config_sampled_pixels(R, strip):
    m, field = strip
    cams = scenes.surround_rig(field, 8)
    ex = scenes.exposure_params(6)
    rr = R.Renderer(19, record_capacity=2_000_000, pair_capacity=12_000_000)
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame(cams)
    rr.forward(st, fr, torch.as_tensor(ex, device="cuda"))
    torch.cuda.synchronize()
    cnt = rr.counts(fr)
    assert cnt.n_records > 300_000 and cnt.n_pairs > 800_000
    pix = sample_pixels(cams, 150, seed=1)
    ref = oracle.render(m, cams, ex, pix)
    assert (ref.T < 0.5).sum() > len(pix) // 3      # the sample does hit the road
    check_pixels(fr, 19, ref, pix)


def test_scene_config_training_step_gradients(R, strip):
    """The bench's training step at full size (1.6M surfels, six 960x540 views,
    16x16 tiles, 2048-key sort chunks; loss fused into the backward, plus the
    grid smoothness term) against the FP64 oracle.  The loss mask holds a
    sample of pixels only, so the exact gradient depends on those pixels alone
    and the oracle computes it by brute force over every surfel.  Sampled
    pixels in the ambiguity band, or with a colour within 1e-3 of its target
    (where the L1 sign could differ between FP32 and FP64), are left out."""
    m, field = strip
    C = 19
    cams = scenes.surround_rig(field, 8)
    ex = scenes.exposure_params(6)
    gi = scenes.grid_index(m)
    tg = scenes.random_targets(cams, C, seed=5)
    pix = np.unique(sample_pixels(cams, 100, seed=4), axis=0)   # each masked pixel once
    ref = oracle.render(m, cams, ex, pix)
    rgb_t, _, _ = oracle.gather_targets(tg, pix)
    keep = (ref.amb == 0) & (np.abs(ref.out[:, :3] - rgb_t).min(1) > 1e-3)
    pix = pix[keep]
    assert len(pix) > 400
    for v in range(len(cams)):
        tg.mask[v][:] = 0
    for v, u, y in pix:
        tg.mask[v][y, u] = 1
    rr = R.Renderer(C, record_capacity=2_000_000, pair_capacity=12_000_000, tile=(16, 16), sort_tile=2048)
    st = R.SurfelTensors.from_map(m, grid_index=gi)
    exd = torch.as_tensor(ex, device="cuda")
    trgb, lab, msk = R.targets_to_device(tg)
    fr = rr.frame(cams)
    loss = torch.empty(1, device="cuda")
    grads = R.zero_grads(st, exd)
    lam = 0.003
    rr.train_step(st, fr, exd, trgb, lab, msk, loss, grads, lambda_smooth=lam)
    torch.cuda.synchronize()
    L, g, _ = oracle.loss_and_grads(m, cams, ex, tg, pix)
    Ls, gs = oracle.smooth_loss(m.xyz[:, 2].astype(np.float64), gi)
    assert abs(loss.item() - (L + lam * Ls)) <= 1e-5 * abs(L + lam * Ls)
    ref_g = g.as_dict()
    ref_g["xyz"] = ref_g["xyz"].copy()
    ref_g["xyz"][:, 2] += lam * gs
    check_gradients({k: v.cpu().numpy().reshape(ref_g[k].shape) for k, v in grads.items()}, ref_g)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_tile_order_is_longest_first_and_stable(R, strip, tile):
    """The compositing kernels take tiles longest list first.  12,240 tiles
    (16x16) are ordered by the one-block counting sort, 48,960 (8x8) by the
    radix pass; both give a permutation in which list lengths fall by at most
    one length class (2^(1/16)) step at a time and equal lengths keep the
    tile index order."""
    m, field = strip
    cams = scenes.surround_rig(field, 8)
    rr = R.Renderer(19, record_capacity=2_000_000, pair_capacity=12_000_000, tile=tile)
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame(cams)
    rr.forward(st, fr, torch.as_tensor(scenes.exposure_params(6), device="cuda"))
    torch.cuda.synchronize()
    cnt = rr.counts(fr)
    T = int(fr.layout.total_tiles)
    assert (T <= 32768) == (tile == (16, 16))
    order = fr.state_section("tile_order", torch.int32, T).cpu().numpy().astype(np.int64)
    _, rg = gpu_tile_lists(fr, cnt)
    length = (rg[:, 1] - rg[:, 0]).clip(min=0)
    np.testing.assert_array_equal(np.sort(order), np.arange(T))
    lo = length[order]
    # classes are floor(16 log2(1 + len)): a later tile is never longer than one class step
    assert np.all(np.log2(1.0 + lo[1:]) <= np.log2(1.0 + lo[:-1]) + 1.0 / 16 + 1e-6)
    assert lo[0] == length.max() or np.log2(1.0 + length.max()) - np.log2(1.0 + lo[0]) < 1.0 / 16
    # equal lengths keep index order: sorting the order by length (stably) must
    # leave the indices of each length ascending
    srt = order[np.argsort(lo, kind="stable")]
    ls = np.sort(lo, kind="stable")
    same = ls[1:] == ls[:-1]
    assert np.all(np.diff(srt)[same] > 0)


def test_batching_config_matches_single_views_and_oracle(R, strip):
    m, field = strip
    cams = []
    for t in range(8):
        cams += scenes.surround_rig(field, 8 + 2 * t, sizes=scenes.BATCH_SIZES)
    assert len(cams) == 48
    ex = scenes.exposure_params(6)
    ext = torch.as_tensor(ex, device="cuda")
    st = R.SurfelTensors.from_map(m)
    rr = R.Renderer(19, record_capacity=12_000_000, pair_capacity=60_000_000)
    fr = rr.frame(cams)
    rr.forward(st, fr, ext)
    torch.cuda.synchronize()
    rr.counts(fr)
    Tb = gpu_state_T(fr)
    r1 = R.Renderer(19, record_capacity=1_000_000, pair_capacity=6_000_000)
    for v in (0, 1, 5, 17, 47):          # single-view renders are bit-identical
        f1 = r1.frame([cams[v]])
        r1.forward(st, f1, ext)
        torch.cuda.synchronize()
        r1.counts(f1)
        assert torch.equal(f1.view(0, 19), fr.view(v, 19))
        c = cams[v]
        np.testing.assert_array_equal(gpu_state_T(f1), Tb[fr.pix_base[v]: fr.pix_base[v] + c.width * c.height])
    sel = [0, 11, 23, 41]
    pix = sample_pixels([cams[v] for v in sel], 60, seed=2, band=False)
    pix_full = pix.copy()
    pix_full[:, 0] = np.array(sel)[pix[:, 0]]
    ref = oracle.render(m, cams, ex, pix_full)
    check_pixels(fr, 19, ref, pix_full)


def test_graph_replay_and_fused_step_equal_the_separate_calls(R):
    """The fused training step (loss inside the backward) and its CUDA-graph
    replay give the forward bit for bit and the loss and gradients of
    rogs_render_fwd + rogs_loss + rogs_render_bwd up to FP32 summation order."""
    m = scenes.tiny_map(C=8)
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 96, res_m=0.06, height_m=20.0)]
    ex = torch.as_tensor(np.array([[0.05, 0.01]], np.float32), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
        st = R.SurfelTensors.from_map(m)
        tg = scenes.random_targets(cams, 8, seed=9)
        trgb, lab, msk = R.targets_to_device(tg)
        fr_e = rr.frame(cams)
        rr.forward(st, fr_e, ex)
        loss_e, g_e = rr.loss(fr_e, trgb, lab, msk)
        grads_e = rr.backward(st, fr_e, ex, g_e)
        # fused, eager
        fr_f = rr.frame(cams)
        loss_f = torch.empty(1, device="cuda")
        grads_f = R.zero_grads(st, ex)
        rr.train_step(st, fr_f, ex, trgb, lab, msk, loss_f, grads_f)
        # fused, graph
        fr_g = rr.frame(cams)
        loss_g = torch.empty(1, device="cuda")
        grads_g = R.zero_grads(st, ex)
        graph = rr.train_graph(st, fr_g, ex, trgb, lab, msk, loss_g, grads_g)
        graph.launch()
        s.synchronize()
        assert torch.equal(fr_g.out, fr_e.out) and torch.equal(fr_f.out, fr_e.out)
        assert abs(loss_g.item() - loss_e.item()) <= 1e-6 * abs(loss_e.item())
        assert abs(loss_f.item() - loss_e.item()) <= 1e-6 * abs(loss_e.item())
        for k in grads_e:
            assert normwise(grads_g[k].cpu().numpy(), grads_e[k].cpu().numpy()) < 1e-5, k
            assert normwise(grads_f[k].cpu().numpy(), grads_e[k].cpu().numpy()) < 1e-5, k
        graph.launch()                     # replays accumulate into the gradients
        s.synchronize()
        assert normwise(grads_g["rgb"].cpu().numpy(), 2 * grads_e["rgb"].cpu().numpy()) < 1e-5
        graph.close()


def test_differentiation_config_crop_gradients(R):
    m, field = scenes.grid_road_map(C=19)
    assert 4_150_000 < m.n < 4_250_000
    cam = scenes.intersection_camera(field)
    cams = [cam]
    ex = np.array([[0.02, -0.01]], np.float32)
    pix = oracle.crop_pixels(0, 288, 296, 64, 64)          # rows 296-359, cols 288-351
    rng = np.random.default_rng(4)
    H, W = cam.height, cam.width
    tg = scenes.Targets([rng.uniform(0, 1, (3, H, W)).astype(np.float32)],
                        [rng.integers(0, 19, (H, W)).astype(np.int32)],
                        [np.ones((H, W), np.uint8)])
    ref = oracle.render(m, cams, ex, pix)
    assert (ref.T < 0.5).mean() > 0.5                      # the crop sees road
    rgb, lb, mk = oracle.gather_targets(tg, pix)
    mk = mk * (ref.amb == 0)
    L, gout = oracle.loss(ref.out, rgb, lb, mk, 19)
    gref = oracle.backward(m, cams, ex, pix, gout)
    rr = R.Renderer(19, record_capacity=2_000_000, pair_capacity=8_000_000)
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame(cams)
    ext = torch.as_tensor(ex, device="cuda")
    rr.forward(st, fr, ext)
    torch.cuda.synchronize()
    rr.counts(fr)
    check_pixels(fr, 19, ref, pix)
    g = rr.backward(st, fr, ext, torch.as_tensor(planar_grad_from_pixels(fr, 19, pix, gout), device="cuda"))
    torch.cuda.synchronize()
    touched = np.nonzero(np.abs(gref.rgb).sum(1))[0]
    assert len(touched) > 50
    check_gradients({k: v.cpu().numpy() for k, v in g.items()}, gref.as_dict())
    # Central finite differences (eps = 1e-4) of the FP64 forward on 512
    # sampled parameters of every type (position, scale, rotation, opacity,
    # colour, logits; exposure too).  The crop's render depends only on the
    # surfels whose footprint reaches it, so the oracle's forward runs on that
    # sub-map (indices keep their order, so depth ties break the same way).
    pr = oracle.project(m, cams)
    kap = 2 * np.log(np.maximum(m.opacity.astype(np.float64), 1e-30) / np.float32(1 / 255))
    rx = np.sqrt(np.maximum(kap * pr.cov[0, :, 0], 0)) + 2.0
    ry = np.sqrt(np.maximum(kap * pr.cov[0, :, 2], 0)) + 2.0
    mx, my = pr.mu[0, :, 0], pr.mu[0, :, 1]
    reach = pr.vis[0] & (mx + rx >= 288) & (mx - rx <= 352) & (my + ry >= 296) & (my - ry <= 360)
    sub = np.nonzero(reach)[0]
    ms = scenes.SurfelMap(m.xyz[sub], m.scale[sub], m.quat[sub], m.opacity[sub], m.rgb[sub], m.sem[sub])
    ok = ref.amb == 0
    pok = pix[ok]
    base = oracle.render(ms, cams, ex, pok)
    assert np.abs(base.out - ref.out[ok]).max() < 1e-12           # the sub-map renders the crop exactly
    tg1 = scenes.Targets(tg.rgb, tg.label, [np.ones((H, W), np.uint8)])
    trgb_ok = oracle.gather_targets(tg1, pok)[0].astype(np.float64)
    rng = np.random.default_rng(5)
    pos = {int(i): j for j, i in enumerate(sub)}
    cand = np.array([i for i in touched if int(i) in pos])
    kinds = [("xyz", 3), ("scale", 2), ("quat", 4), ("opacity", 1), ("rgb", 3), ("sem", 19)]
    eps = 1e-4
    rows, flips = [], 0
    gnp = {k: v.cpu().numpy().reshape(v.shape[0], -1) for k, v in g.items()}
    smp = 0
    got = {k: 0 for k, _ in kinds}
    while len(rows) < 512 and smp < 3000:          # 512 compared samples, types in equal shares
        if smp < 2:                                   # the camera's exposure (a, b)
            name, i, kk = "exposure", 0, smp
        else:
            name, width = min(kinds, key=lambda kw: got[kw[0]])
            i, kk = int(rng.choice(cand)), int(rng.integers(0, width))
        smp += 1
        vals, flip = [], False
        for d in (eps, -eps):
            mp, exp_ = ms.copy(), ex.astype(np.float64).copy()
            if name == "exposure":
                exp_[0, kk] += d
            else:
                arr = getattr(mp, name).astype(np.float64)
                arr.reshape(ms.n, -1)[pos[i], kk] += d
                setattr(mp, name, arr)
            Lp, rp = oracle.loss_value(mp, cams, exp_, tg1, pok)
            flip |= not np.array_equal(rp.sig, base.sig)   # a composited list changed: discontinuity
            # an exposed colour crossing its target: the L1 kink is inside [-eps, eps]
            flip |= bool((np.sign(rp.out[:, :3] - trgb_ok) != np.sign(base.out[:, :3] - trgb_ok)).any())
            vals.append(Lp)
        if flip:
            flips += 1
            continue
        fd = (vals[0] - vals[1]) / (2 * eps)
        gpu = float(gnp[name][i, kk])
        rows.append((name, fd, gpu))
        if name in got:
            got[name] += 1
    # samples whose perturbation changes a composited list (an alpha crossing
    # alpha_min at some crop pixel: common for the large near-camera
    # footprints' geometry) or moves a colour across its L1 target are left
    # out, counted and replaced by new draws
    assert len(rows) == 512 and flips <= 0.75 * smp, (len(rows), flips, smp)
    fd = np.array([r[1] for r in rows]); gg = np.array([r[2] for r in rows])
    assert np.abs(fd - gg).max() <= 1e-3 * np.abs(fd).max(), (np.abs(fd - gg).max(), np.abs(fd).max())
    for name, _ in kinds:                    # and per parameter type, against that type's scale
        sel = np.array([r[0] == name for r in rows])
        assert sel.sum() >= 40, (name, sel.sum())
        assert np.abs(fd[sel] - gg[sel]).max() <= 1e-3 * np.abs(fd[sel]).max(), name
    print(f"finite differences: {len(rows)} samples compared, {flips} draws left out (a list or an L1 sign changed)")
