"""CUDA path vs the FP64 oracle, through the C-ABI (small and ragged cases).

Tolerances (spec contract): bit-exact for sort order and tile lists;
1e-4 max-abs for rendered rgb and semantics, depth relative to the view's
depth scale; 1e-3 relative for gradients, normwise and element-wise with a
floor (tests/_util.py: check_gradients).  Pixels inside the
ambiguity band (some surfel's alpha*g within 2e-5 relative of alpha_min, or a
transmittance step within 1e-4 relative of t_min) are excluded and counted;
the count must stay below 0.01 % of the pixels (or a handful on tiny frames).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _util import (check_gradients, gpu_pixels, gpu_records, gpu_rects, gpu_state_T, gpu_tile_lists,  # noqa: E402
                   normwise, pixel_index, planar_grad_from_pixels)

TOL_RGB = 1e-4


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render
    return render


def make(R, C, tile=(16, 16), rec=1 << 18, pairs=1 << 21):
    return R.Renderer(C, record_capacity=rec, pair_capacity=pairs, tile=tile)


def gpu_render(R, rr, m, cams, ex):
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame(cams)
    ext = torch.as_tensor(np.asarray(ex, np.float32), device="cuda")
    rr.forward(st, fr, ext)
    torch.cuda.synchronize()
    cnt = rr.counts(fr)
    return st, fr, ext, cnt


def compare_forward(R, rr, m, cams, ex, depth_scale, max_band_frac=1e-4, max_band_abs=8):
    st, fr, ext, cnt = gpu_render(R, rr, m, cams, ex)
    pix = oracle.full_pixels(cams)
    ref = oracle.render(m, cams, ex, pix)
    got = gpu_pixels(fr, m.num_classes, pix)
    band = ref.amb != 0
    n_band = int(band.sum())
    assert n_band <= max(max_band_abs, max_band_frac * len(pix)), n_band
    ok = ~band
    C = m.num_classes
    e_rgb = np.abs(got[ok, :3] - ref.out[ok, :3]).max()
    e_sem = np.abs(got[ok, 3:3 + C] - ref.out[ok, 3:3 + C]).max() if C else 0.0
    dsc = np.array([depth_scale[v] for v in pix[ok, 0]])
    e_dep = (np.abs(got[ok, 3 + C] - ref.out[ok, 3 + C]) / dsc).max()
    T = gpu_state_T(fr)[pixel_index(fr, pix)]
    e_T = np.abs(T[ok] - ref.T[ok]).max()
    assert e_rgb < TOL_RGB, e_rgb
    assert e_sem < TOL_RGB, e_sem
    assert e_dep < TOL_RGB, e_dep
    assert e_T < TOL_RGB, e_T
    # E, the composited (pixel, surfel) pairs the forward counts, against the
    # oracle's per-pixel counts: equal unless a pixel sits in the ambiguity
    # band, where a threshold or stop decision may go either way
    e_ref = int(ref.ncomp.sum())
    if n_band == 0:
        assert int(cnt.composited) == e_ref
    else:
        assert abs(int(cnt.composited) - e_ref) <= 64 * n_band, (int(cnt.composited), e_ref, n_band)
    return st, fr, ext, cnt, ref, pix


# ---------------------------------------------------------------- sort

@pytest.mark.parametrize("sort_tile", [1024, 2048, 4096, 8192])
@pytest.mark.parametrize("n,bits", [(1, 32), (4095, 8), (4096, 18), (4097, 32), (123457, 18), (1 << 20, 32),
                                    (250001, 5), (1999999, 24)])
def test_radix_sort_is_stable_and_exact(R, n, bits, sort_tile):
    rr = R.Renderer(0, record_capacity=1 << 10, pair_capacity=1 << 21, sort_tile=sort_tile)
    rng = np.random.default_rng(n)
    hi = (1 << bits) - 1
    keys = rng.integers(0, hi + 1, size=n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 3] = keys[n // 3: 2 * (n // 3)] if n > 3 else keys[: n // 3]   # many duplicates
    vals = np.arange(n, dtype=np.uint32)
    kt = torch.as_tensor(keys.view(np.int32), device="cuda")
    vt = torch.as_tensor(vals.view(np.int32), device="cuda")
    ko, vo = rr.sort_pairs(kt, vt, bits)
    order = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    np.testing.assert_array_equal(vo.cpu().numpy().view(np.uint32), vals[order])
    # input untouched
    np.testing.assert_array_equal(kt.cpu().numpy().view(np.uint32), keys)


def test_radix_sort_empty(R):
    rr = make(R, 0)
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    ko, vo = rr.sort_pairs(e, e, 32)
    assert ko.numel() == 0


# ---------------------------------------------------------- projection

def test_records_match_oracle_projection(R):
    m = scenes.tiny_map()
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.1, 3.2), 96, res_m=0.05, height_m=20.0)]
    cams[1].exposure_idx = 1
    rr = make(R, m.num_classes)
    ex = np.zeros((2, 2), np.float32)
    st, fr, ext, cnt = gpu_render(R, rr, m, cams, ex)
    rec = gpu_records(fr, cnt)
    pr = oracle.project(m, cams)
    assert cnt.n_records == len(rec) > 1000
    v = rec["view"].astype(np.int64); s = rec["surfel"].astype(np.int64)
    # every record is oracle-visible and records are in (view, surfel) order
    assert pr.vis[v, s].all()
    key = v * m.n + s
    assert (np.diff(key) > 0).all()
    mu = np.stack([rec["mxi"].astype(np.float64) + rec["mxf"], rec["myi"].astype(np.float64) + rec["myf"]], -1)
    assert np.abs(mu - pr.mu[v, s]).max() < 2e-5
    assert ((rec["mxf"] >= 0) & (rec["mxf"] <= 1) & (rec["myf"] >= 0) & (rec["myf"] <= 1)).all()
    con = np.stack([rec["ca"], rec["cb"], rec["cc"]], -1).astype(np.float64)
    scale = np.abs(pr.con[v, s]).max(-1, keepdims=True)
    assert (np.abs(con - pr.con[v, s]) / scale).max() < 1e-5
    assert (np.abs(rec["depth"] - pr.depth[v, s]) / np.abs(pr.depth[v, s])).max() < 1e-6
    # the binary32 sort key is bit-identical
    np.testing.assert_array_equal(rec["key"].view(np.uint32), pr.key[v, s].view(np.uint32))
    # oracle-visible surfels without a record lie outside the image (conservative footprint)
    have = np.zeros_like(pr.vis)
    have[v, s] = True
    miss_v, miss_s = np.nonzero(pr.vis & ~have)
    kappa = 2 * np.log(m.opacity[miss_s] / np.float32(1 / 255))
    rx = np.sqrt(kappa * pr.cov[miss_v, miss_s, 0]); ry = np.sqrt(kappa * pr.cov[miss_v, miss_s, 2])
    mx = pr.mu[miss_v, miss_s, 0]; my = pr.mu[miss_v, miss_s, 1]
    W = np.array([c.width for c in cams])[miss_v]; H = np.array([c.height for c in cams])[miss_v]
    outside = (mx + rx < 0.5) | (mx - rx > W - 0.5) | (my + ry < 0.5) | (my - ry > H - 0.5)
    assert outside.all()


def test_box_cull_matches_hand_worked_geometry(R):
    """The kernels' perspective box cull against the hand-worked ground boxes of
    the oracle pins (supplementary box cull): every record's surfel lies in its
    camera's box, and every surfel in the box without a record has a footprint
    entirely off the image."""
    import test_oracle_box as box
    for yaw, pitch, roll, cxy in box.CASES:
        xh, zh = box.hand_ground_axes(yaw, pitch, roll)
        m, LF, keep = box.box_map(cxy, xh, zh)
        cam = box.box_camera(yaw, pitch, roll, cxy)
        rr = make(R, m.num_classes)
        st, fr, ext, cnt = gpu_render(R, rr, m, [cam], np.zeros((1, 2)))
        rec = gpu_records(fr, cnt)
        s = rec["surfel"].astype(np.int64)
        assert keep[s].all(), [tuple(LF[i]) for i in s[~keep[s]]]
        pr = oracle.project(m, [cam])
        have = np.zeros(m.n, bool)
        have[s] = True
        miss = np.nonzero(keep & ~have)[0]
        kappa = 2 * np.log(m.opacity[miss] / np.float32(1 / 255))
        rx = np.sqrt(kappa * pr.cov[0, miss, 0]); ry = np.sqrt(kappa * pr.cov[0, miss, 2])
        mx = pr.mu[0, miss, 0]; my = pr.mu[0, miss, 1]
        outside = (mx + rx < 0.5) | (mx - rx > cam.width - 0.5) | (my + ry < 0.5) | (my - ry > cam.height - 0.5)
        assert outside.all()
        assert len(s) >= 8   # the box's far part is on the image
        rr.close()


def test_tile_lists_are_bit_exact(R):
    m = scenes.tiny_map()
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.1, 3.2), 100, res_m=0.05, height_m=20.0)]
    for tile in [(16, 16), (32, 8), (8, 8)]:
        rr = make(R, m.num_classes, tile=tile)
        st, fr, ext, cnt = gpu_render(R, rr, m, cams, np.zeros((1, 2)))
        rec = gpu_records(fr, cnt)
        rect = gpu_rects(fr, cnt)
        nonempty = (rect[:, 2] >= rect[:, 0]) & (rect[:, 3] >= rect[:, 1])
        tx = [-(-c.width // tile[0]) for c in cams]; ty = [-(-c.height // tile[1]) for c in cams]
        tb = np.concatenate([[0], np.cumsum(np.array(tx) * np.array(ty))[:-1]])
        T = int(sum(a * b for a, b in zip(tx, ty)))
        ids = np.nonzero(nonempty)[0]
        offs, lst = oracle.binning(rect[ids], rec["view"][ids], rec["key"][ids], rec["surfel"][ids].astype(np.int64),
                                   tb, tx, T)
        pr, rg = gpu_tile_lists(fr, cnt)
        assert cnt.n_pairs == offs[-1]
        for t in range(T):
            mine = pr[rg[t, 0]:rg[t, 1]] if rg[t, 1] > rg[t, 0] else np.zeros(0, np.int64)
            np.testing.assert_array_equal(mine, ids[lst[offs[t]:offs[t + 1]]])


def test_long_tile_lists_are_exact(R):
    """Lists of 10,000 entries per tile (several sort chunks): a dense flat
    patch of equal depths, so the order is decided by the surfel index alone,
    seen by a small orthographic camera whose every tile holds every surfel;
    the lists equal the integer binning reference and the forward (which
    walks the whole list to the transmittance stop) matches the oracle."""
    n1 = 100
    g = (np.arange(n1) * 0.012).astype(np.float32)
    xx, yy = np.meshgrid(g, g)
    n = n1 * n1
    rng = np.random.default_rng(8)
    m = scenes.SurfelMap(xyz=np.stack([xx.ravel(), yy.ravel(), np.zeros(n)], -1).astype(np.float32),
                         scale=np.full((n, 2), 0.3, np.float32),     # every footprint covers all four tiles
                         quat=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                         opacity=np.full(n, 0.05, np.float32), rgb=rng.uniform(0, 1, (n, 3)).astype(np.float32),
                         sem=rng.normal(0, 1, (n, 2)).astype(np.float32))
    cam = scenes.bev_camera((0.6, 0.6), 32, res_m=0.05, height_m=10.0)
    rr = make(R, 2, rec=1 << 15, pairs=1 << 17)
    st, fr, ext, cnt = gpu_render(R, rr, m, [cam], np.zeros((1, 2)))
    rec = gpu_records(fr, cnt)
    rect = gpu_rects(fr, cnt)
    pr, rg = gpu_tile_lists(fr, cnt)
    lens = rg[:, 1] - rg[:, 0]
    assert lens.min() == n, lens
    ids = np.arange(len(rec))
    offs, lst = oracle.binning(rect, rec["view"], rec["key"], rec["surfel"].astype(np.int64), [0], [2], 4)
    assert cnt.n_pairs == offs[-1]
    for t in range(4):
        np.testing.assert_array_equal(pr[rg[t, 0]:rg[t, 1]], ids[lst[offs[t]:offs[t + 1]]])
    # every pixel here composits until the transmittance stop, so more of them
    # sit in the stop's ambiguity band than in a road scene
    compare_forward(R, rr, m, [cam], np.zeros((1, 2), np.float32), depth_scale=[10.0], max_band_abs=24)


# ------------------------------------------------------------- forward

def test_forward_tiny_matches_oracle(R):
    m = scenes.tiny_map()
    cam = scenes.tiny_camera()
    for tile in [(16, 16), (32, 8), (8, 8)]:
        rr = make(R, m.num_classes, tile=tile)
        compare_forward(R, rr, m, [cam], np.array([[0.1, -0.03]], np.float32), depth_scale=[40.0])


def test_schedule_choices_do_not_change_the_forward(R):
    """The sort chunk only reorders work: outputs are bit-identical.  The tile
    shape changes which entries a warp stages, but every pixel still adds the
    same contributions in the same depth order with the same fused
    multiply-adds (entries that do not reach it add an exact zero), so the
    channels and the transmittance are bit-identical too (the last
    contributor is a position in the tile's own list, so it is compared only
    across sort chunks)."""
    m = scenes.tiny_map(C=5)
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 77, res_m=0.05, height_m=20.0)]
    ex = np.zeros((1, 2), np.float32)
    ref = None
    for tile in [(16, 16), (32, 8), (8, 8)]:
        by_chunk = None
        for st_ in (2048, 8192):
            rr = R.Renderer(5, record_capacity=1 << 16, pair_capacity=1 << 20, tile=tile, sort_tile=st_)
            st, fr, ext, cnt = gpu_render(R, rr, m, cams, ex)
            P = fr.layout.total_pixels
            res = (fr.out.cpu().numpy(), gpu_state_T(fr),
                   fr.state_section("pix_last", torch.int32, P).cpu().numpy())
            if by_chunk is None:
                by_chunk = res
            else:
                for x, y in zip(res, by_chunk):
                    np.testing.assert_array_equal(x, y)
        if ref is None:
            ref = by_chunk
        else:
            np.testing.assert_array_equal(by_chunk[1], ref[1])
            np.testing.assert_array_equal(by_chunk[0], ref[0])


def test_forward_ragged_multiview_and_ortho(R):
    m = scenes.tiny_map(C=3)
    c0 = scenes.tiny_camera()
    c1 = scenes.make_camera(scenes.PERSP, 37, 23, 30.0, 30.0, scenes.look_rotation(5.0, 25.0), (-1.0, 3.0, 1.2),
                            exposure_idx=1, use_box_cull=0)
    c2 = scenes.bev_camera((3.0, 3.0), 130, res_m=0.05, height_m=30.0, exposure_idx=2)
    c3 = scenes.bev_camera((1.0, 5.5), 17, res_m=0.2, height_m=10.0, exposure_idx=0)
    cams = [c0, c1, c2, c3]
    ex = np.array([[0.0, 0.0], [0.2, 0.01], [-0.1, 0.05]], np.float32)
    rr = make(R, m.num_classes, tile=(16, 16))
    compare_forward(R, rr, m, cams, ex, depth_scale=[40.0, 40.0, 30.0, 10.0])


def test_flat_road_ortho_ties_break_by_index(R):
    """All depths bit-equal: ordering falls to the surfel index everywhere."""
    m = scenes.tiny_map(C=2)
    m.xyz[:, 2] = 0.0
    m.quat[:] = np.array([1, 0, 0, 0], np.float32)
    m.scale[:] = 0.09
    cam = scenes.bev_camera((3.15, 3.15), 160, res_m=0.04, height_m=25.0)
    rr = make(R, 2)
    compare_forward(R, rr, m, [cam], np.zeros((1, 2)), depth_scale=[25.0])


def test_empty_and_all_culled(R):
    m = scenes.tiny_map(C=2)
    sky = scenes.make_camera(scenes.PERSP, 64, 48, 50.0, 50.0, scenes.look_rotation(180.0, -30.0), (-2.0, 3.0, 1.5))
    rr = make(R, 2)
    st, fr, ext, cnt = gpu_render(R, rr, m, [sky], np.array([[0.3, 0.25]], np.float32))
    assert cnt.n_records == 0 and cnt.n_pairs == 0
    out = fr.view(0, 2).cpu().numpy()
    np.testing.assert_allclose(out[:3], 0.25, atol=1e-7)      # background 0 -> exposure b
    assert np.abs(out[3:]).max() == 0
    np.testing.assert_array_equal(gpu_state_T(fr), 1.0)
    # an empty map
    e = scenes.SurfelMap(np.zeros((0, 3), np.float32), np.zeros((0, 2), np.float32), np.zeros((0, 4), np.float32),
                         np.zeros(0, np.float32), np.zeros((0, 3), np.float32), np.zeros((0, 2), np.float32))
    st, fr, ext, cnt = gpu_render(R, rr, e, [scenes.tiny_camera()], np.zeros((1, 2)))
    assert cnt.n_records == 0
    assert np.abs(fr.view(0, 2).cpu().numpy()).max() == 0


def test_capacity_overflow_is_reported(R):
    from paper_2405_14342_gb300 import rogs
    m = scenes.tiny_map()
    rr = make(R, m.num_classes, rec=500, pairs=900)
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame([scenes.tiny_camera()])
    rr.forward(st, fr, torch.zeros(1, 2, device="cuda"))
    torch.cuda.synchronize()
    with pytest.raises(rogs.RogsError) as ei:
        rr.counts(fr)
    assert ei.value.status == rogs.ROGS_ERR_CAPACITY
    c = rr.counts(fr, check=False)
    assert c.need_records > 500 and c.n_records == 500 and c.status & 1
    # a context with room renders the same cameras fine afterwards, in a frame
    # laid out for its own capacities (the small context's frame is refused)
    rr2 = make(R, m.num_classes)
    with pytest.raises(ValueError, match="another Renderer"):
        rr2.forward(st, fr, torch.zeros(1, 2, device="cuda"))
    fr2 = rr2.frame([scenes.tiny_camera()])
    rr2.forward(st, fr2, torch.zeros(1, 2, device="cuda"))
    torch.cuda.synchronize()
    assert rr2.counts(fr2).status == 0


def test_invalid_arguments_are_rejected(R):
    from paper_2405_14342_gb300 import rogs
    m = scenes.tiny_map(C=2)
    rr = make(R, 2)
    st = R.SurfelTensors.from_map(m)
    cam = scenes.tiny_camera()
    fr = rr.frame([cam])
    bad = scenes.tiny_camera(); bad.exposure_idx = 3
    with pytest.raises(rogs.RogsError) as ei:
        rr.forward(st, rr.frame([bad]), torch.zeros(1, 2, device="cuda"))
    assert ei.value.status == rogs.ROGS_ERR_INVALID
    with pytest.raises(rogs.RogsError):
        rogs.rogs_render_fwd(rr.ctx, st.c_struct(), fr.cam_arr, 0, torch.zeros(1, 2, device="cuda"), fr.out,
                             fr.state)
    bad2 = scenes.tiny_camera(); bad2.fx = -1.0
    with pytest.raises(rogs.RogsError):
        rr.frame([bad2])
    with pytest.raises(rogs.RogsError):
        R.Renderer(2, tile=(12, 12))


# ---------------------------------------------------------------- loss

def test_loss_kernel_matches_oracle_loss(R):
    m = scenes.tiny_map()
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 64, res_m=0.1, height_m=20.0)]
    rr = make(R, m.num_classes)
    st, fr, ext, cnt = gpu_render(R, rr, m, cams, np.zeros((1, 2)))
    tg = scenes.random_targets(cams, m.num_classes, seed=4)
    trgb, lab, msk = R.targets_to_device(tg)
    loss, gout = rr.loss(fr, trgb, lab, msk, 1.0, 0.06)
    torch.cuda.synchronize()
    pix = oracle.full_pixels(cams)
    out = gpu_pixels(fr, m.num_classes, pix)
    rgb, lb, mk = oracle.gather_targets(tg, pix)
    L, g = oracle.loss(out, rgb, lb, mk, m.num_classes)
    assert abs(float(loss.item()) - L) < 1e-5 * max(1.0, abs(L))
    gg = planar_grad_from_pixels(fr, m.num_classes, pix, g)
    got = gout.cpu().numpy()
    assert np.abs(got - gg).max() < 1e-9 + 1e-5 * np.abs(gg).max()


def test_loss_empty_mask(R):
    m = scenes.tiny_map(C=2)
    cams = [scenes.tiny_camera()]
    rr = make(R, 2)
    st, fr, ext, cnt = gpu_render(R, rr, m, cams, np.zeros((1, 2)))
    tg = scenes.random_targets(cams, 2, mask_frac=0.0)
    trgb, lab, msk = R.targets_to_device(tg)
    loss, gout = rr.loss(fr, trgb, lab, msk)
    torch.cuda.synchronize()
    assert loss.item() == 0.0 and gout.abs().max().item() == 0.0


# ------------------------------------------------------------ backward

def _generic_tiny(C=8):
    m = scenes.tiny_map(C=C)
    g = np.random.default_rng(3)
    m.scale = (0.06 * g.uniform(0.7, 1.3, size=(m.n, 2))).astype(np.float32)
    th = g.uniform(0, 2 * np.pi, m.n)
    q = m.quat.astype(np.float64)
    w1, x1, y1, z1 = q.T
    w2, z2 = np.cos(th / 2), np.sin(th / 2)
    m.quat = (np.stack([w1 * w2 - z1 * z2, x1 * w2 + y1 * z2, y1 * w2 - x1 * z2, w1 * z2 + z1 * w2], -1)
              * g.uniform(0.8, 1.2, size=(m.n, 1))).astype(np.float32)
    m.opacity = g.uniform(0.5, 0.995, size=m.n).astype(np.float32)
    return m


def compare_backward(R, rr, m, cams, ex, tg, pix_sel=None, tol=1e-3):
    st, fr, ext, cnt = gpu_render(R, rr, m, cams, ex)
    pix = oracle.full_pixels(cams) if pix_sel is None else pix_sel
    ref = oracle.render(m, cams, ex, pix)
    rgb, lb, mk = oracle.gather_targets(tg, pix)
    mk = mk * (ref.amb == 0)            # the ambiguity band is left out of the loss
    L, gout = oracle.loss(ref.out, rgb, lb, mk, m.num_classes)
    gref = oracle.backward(m, cams, ex, pix, gout)
    gpl = torch.as_tensor(planar_grad_from_pixels(fr, m.num_classes, pix, gout), device="cuda")
    g = rr.backward(st, fr, ext, gpl)
    torch.cuda.synchronize()
    return check_gradients({k: v.cpu().numpy() for k, v in g.items()}, gref.as_dict())


def test_backward_tiny_matches_oracle(R):
    m = _generic_tiny()
    cams = [scenes.tiny_camera()]
    tg = scenes.random_targets(cams, m.num_classes, seed=5)
    for tile in [(16, 16), (32, 8), (8, 8)]:
        rr = make(R, m.num_classes, tile=tile)
        compare_backward(R, rr, m, cams, np.array([[0.1, -0.02]], np.float32), tg)


def test_backward_multiview_ortho_and_wide_classes(R):
    m = _generic_tiny(C=23)     # 64-channel gradient rows
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 96, res_m=0.06, height_m=25.0, exposure_idx=1)]
    tg = scenes.random_targets(cams, m.num_classes, seed=6)
    rr = make(R, m.num_classes)
    compare_backward(R, rr, m, cams, np.array([[0.05, 0.0], [-0.1, 0.02]], np.float32), tg)


def test_backward_is_repeatable_and_buffer_clears(R):
    m = _generic_tiny(C=4)
    cams = [scenes.tiny_camera()]
    rr = make(R, 4)
    st, fr, ext, cnt = gpu_render(R, rr, m, cams, np.zeros((1, 2)))
    gout = torch.randn_like(fr.out) * 1e-3
    g1 = rr.backward(st, fr, ext, gout)
    g2 = rr.backward(st, fr, ext, gout)
    torch.cuda.synchronize()
    for k in g1:
        a, b = g1[k].cpu().numpy(), g2[k].cpu().numpy()
        assert normwise(a, b) < 1e-5, k


# ---------------------------------------------------------------- init

def test_init_from_poses_matches_oracle(R):
    rng = np.random.default_rng(9)
    P = 300
    poses = np.zeros((P, 12), np.float32)
    for k in range(P):
        yaw, roll, pitch = rng.uniform(-np.pi, np.pi), rng.normal(0, 0.05), rng.normal(0, 0.05)
        cz, sz = math.cos(yaw), math.sin(yaw)
        Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
        Rx = np.array([[1, 0, 0], [0, math.cos(roll), -math.sin(roll)], [0, math.sin(roll), math.cos(roll)]])
        Ry = np.array([[math.cos(pitch), 0, math.sin(pitch)], [0, 1, 0], [-math.sin(pitch), 0, math.cos(pitch)]])
        poses[k, :3] = (rng.uniform(0, 400), rng.uniform(0, 40), rng.normal(0, 0.3))
        poses[k, 3:] = (Rz @ Ry @ Rx).ravel()
    x, y = scenes.grid_xy(400, 40, spacing=1.0)
    xy = np.stack([x, y], -1).astype(np.float32)
    rr = make(R, 0)
    for exact in (True, False):
        z, q, near = rr.init_from_poses(torch.as_tensor(xy, device="cuda"), poses, exact_plane=exact)
        rc, zr, Rr, nr = oracle.init_from_poses(xy, poses, exact_plane=exact)
        np.testing.assert_array_equal(near.cpu().numpy(), nr)
        assert np.abs(z.cpu().numpy() - zr).max() < 2e-5
        qq = q.cpu().numpy().astype(np.float64)
        assert (qq[:, 0] >= 0).all()
        w, a, b, c = qq.T
        Rq = np.stack([1 - 2 * (b * b + c * c), 2 * (a * b - w * c), 2 * (a * c + w * b),
                       2 * (a * b + w * c), 1 - 2 * (a * a + c * c), 2 * (b * c - w * a),
                       2 * (a * c - w * b), 2 * (b * c + w * a), 1 - 2 * (a * a + b * b)], -1).reshape(-1, 3, 3)
        assert np.abs(Rq - Rr).max() < 2e-6


def test_init_rejects_degenerate_pose(R):
    from paper_2405_14342_gb300 import rogs
    rr = make(R, 0)
    poses = np.zeros((1, 12), np.float32)
    poses[0, 3:] = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], np.float32).ravel()
    with pytest.raises(rogs.RogsError) as ei:
        rr.init_from_poses(torch.zeros(4, 2, device="cuda"), poses, exact_plane=True)
    assert ei.value.status == rogs.ROGS_ERR_INVALID


def test_extreme_class_counts(R):
    """No semantic classes (8 padded channels) and 40 classes (64 padded
    channels, the widest kernels): forward and backward against the oracle."""
    cams = [scenes.tiny_camera()]
    for C in (0, 40):
        m = _generic_tiny(C=C)
        rr = make(R, C)
        compare_forward(R, rr, m, cams, np.zeros((1, 2), np.float32), depth_scale=[40.0])
        tg = scenes.random_targets(cams, C, seed=8)
        compare_backward(R, make(R, C), m, cams, np.array([[0.05, 0.01]], np.float32), tg)
