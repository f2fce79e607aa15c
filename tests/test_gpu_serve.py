"""Serving loop (rogs_serve_*): results vs the FP64 oracle, the same result
alone and in a mix of concurrent requests, admission errors, and continuous
batching actually batching."""
import math
import time

import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render, rogs, serve
    m = scenes.tiny_map(C=8)
    st = render.SurfelTensors.from_map(m)
    ex_np = np.array([[0.05, -0.02], [0.0, 0.0]], np.float32)
    ex = torch.as_tensor(ex_np, device="cuda")
    cfg = rogs.rogs_default_config(8, 1 << 18, 1 << 21)
    return dict(render=render, rogs=rogs, serve=serve, m=m, st=st, ex=ex, ex_np=ex_np, cfg=cfg)


def requests():
    cams = [
        (scenes.bev_camera((3.1, 3.1), 64, res_m=0.1, height_m=30.0, exposure_idx=0), 7),
        (scenes.tiny_camera(), 7),
        (scenes.bev_camera((1.5, 4.0), 40, res_m=0.05, height_m=10.0, exposure_idx=1), 1),
        (scenes.make_camera(scenes.PERSP, 96, 54, 60.0, 60.0, scenes.look_rotation(10.0, 15.0), (-1.0, 3.0, 1.2),
                            exposure_idx=1, use_box_cull=1), 6),
        (scenes.bev_camera((4.0, 2.0), 33, res_m=0.07, height_m=12.0, exposure_idx=0), 2),
    ]
    return cams


def test_serve_results_match_oracle(env):
    srv = env["serve"].Server(env["cfg"], env["st"], env["ex"], max_batch_views=8, max_inflight=2,
                              memory_budget=1 << 30, record_capacity=1 << 18, pair_capacity=1 << 21)
    try:
        reqs = requests()
        tickets = [srv.submit(c, ch) for c, ch in reqs]
        res = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    m = env["m"]
    for (cam, ch), r in zip(reqs, res):
        pix = oracle.full_pixels([cam])
        ref = oracle.render(m, [cam], env["ex_np"], pix)
        H, W = cam.height, cam.width
        ok = (ref.amb == 0).reshape(H, W)
        out = ref.out.reshape(H, W, -1)
        if ch & 1:
            assert np.abs(r["rgb"].transpose(1, 2, 0)[ok] - out[ok][:, :3]).max() < 1e-4
        if ch & 4:
            cov = 1.0 - ref.T.reshape(H, W)
            R64 = cam.R.astype(np.float64)
            cam_z = -(R64.T @ cam.t.astype(np.float64))[2]
            D = out[..., 3 + m.num_classes]
            with np.errstate(divide="ignore", invalid="ignore"):
                exp = np.where(cov >= 0.5, (cam_z - D / cov) if cam.kind == scenes.ORTHO else D / cov, np.nan)
            sure = ok & (np.abs(cov - 0.5) > 1e-4)
            assert np.array_equal(np.isnan(r["elev"][sure]), np.isnan(exp[sure]))
            fin = sure & ~np.isnan(exp)
            assert np.abs(r["elev"][fin] - exp[fin]).max() < 1e-3
        if ch & 2:
            logits = out[..., 3:3 + m.num_classes]
            top2 = np.sort(logits, -1)[..., -2:]
            clear = ok & (top2[..., 1] - top2[..., 0] > 1e-4)
            np.testing.assert_array_equal(r["sem"][clear], logits.argmax(-1)[clear])


def test_result_alone_equals_result_in_a_mix(env):
    reqs = requests()
    srv1 = env["serve"].Server(env["cfg"], env["st"], env["ex"], max_batch_views=1, max_inflight=1,
                               memory_budget=1 << 30, record_capacity=1 << 18, pair_capacity=1 << 21)
    try:
        alone = [srv1.wait(srv1.submit(c, ch)) for c, ch in reqs]
    finally:
        srv1.close()
    srv = env["serve"].Server(env["cfg"], env["st"], env["ex"], max_batch_views=16, max_inflight=3,
                              memory_budget=1 << 30, record_capacity=1 << 18, pair_capacity=1 << 22)
    try:
        mix = reqs * 4
        rng = np.random.default_rng(0)
        order = rng.permutation(len(mix))
        tickets = {}
        # three large requests first keep every stream busy for a few
        # milliseconds, so the mix arrives while nothing is free and is batched
        busy = [srv.submit(scenes.bev_camera((3.1, 3.1), 2048, res_m=0.004, height_m=30.0), 7) for _ in range(3)]
        for i in order:
            c, ch = mix[i]
            tickets[i] = srv.submit(c, ch)
        results = {i: srv.wait(t) for i, t in tickets.items()}
        for t in busy:
            srv.wait(t)
        st = srv.stats()
        assert st.completed == len(mix) + 3 and st.failed == 0
        assert st.batches < len(mix)                      # requests were batched
    finally:
        srv.close()
    for i, r in results.items():
        a = alone[i % len(reqs)]
        for k in a:
            np.testing.assert_array_equal(r[k], a[k])     # bit for bit, NaNs included


def test_admission_errors(env):
    rogs = env["rogs"]
    srv = env["serve"].Server(env["cfg"], env["st"], env["ex"], max_batch_views=4, max_inflight=1, max_queue=2,
                              memory_budget=64 << 20, record_capacity=1 << 16, pair_capacity=1 << 18)
    try:
        huge = scenes.bev_camera((3.0, 3.0), 4096, res_m=0.01, height_m=10.0)
        with pytest.raises(rogs.RogsError) as ei:
            srv.submit(huge, 7)
        assert ei.value.status == rogs.ROGS_ERR_OOM
        bad = scenes.tiny_camera()
        bad.exposure_idx = 9
        with pytest.raises(rogs.RogsError) as ei:
            srv.submit(bad, 1)
        assert ei.value.status == rogs.ROGS_ERR_INVALID
        with pytest.raises(rogs.RogsError) as ei:
            srv.submit(scenes.tiny_camera(), 0)
        assert ei.value.status == rogs.ROGS_ERR_INVALID
        # the queue bound: keep submitting until BUSY shows up (pending requests only)
        busy = False
        tickets = []
        for _ in range(64):
            try:
                tickets.append(srv.submit(scenes.tiny_camera(), 1))
            except rogs.RogsError as e:
                assert e.status == rogs.ROGS_ERR_BUSY
                busy = True
                break
        assert busy
        for t in tickets:
            srv.wait(t)
        with pytest.raises(rogs.RogsError):
            srv.poll(tickets[0]) if tickets[0] in srv._meta else rogs.rogs_serve_poll(srv.h, tickets[0], None)
    finally:
        srv.close()


def test_serve_timeout_is_reported_and_the_server_keeps_serving(env):
    """A batch still running after timeout_s fails its requests with
    ROGS_ERR_TIMEOUT (the host stops waiting; the GPU work itself finishes and
    its memory is released then); with a longer timeout the same server then
    serves new requests correctly."""
    rogs = env["rogs"]
    srv = env["serve"].Server(env["cfg"], env["st"], env["ex"], max_batch_views=1, max_inflight=1,
                              memory_budget=4 << 30, record_capacity=1 << 18, pair_capacity=1 << 23,
                              timeout_s=1e-6)
    try:
        big = scenes.bev_camera((3.1, 3.1), 4096, res_m=0.002, height_m=30.0)   # 16.8 Mpx, 285 MB of result
        t = srv.submit(big, 7)
        with pytest.raises(rogs.RogsError) as ei:
            srv.wait(t, timeout=60.0)
        assert ei.value.status == rogs.ROGS_ERR_TIMEOUT
        assert srv.stats().failed == 1
        srv.set_timeout(30.0)
        cam, ch = requests()[1]
        r = srv.wait(srv.submit(cam, ch))
    finally:
        srv.close()
    pix = oracle.full_pixels([cam])
    ref = oracle.render(env["m"], [cam], env["ex_np"], pix)
    ok = (ref.amb == 0).reshape(cam.height, cam.width)
    out = ref.out.reshape(cam.height, cam.width, -1)
    assert np.abs(r["rgb"].transpose(1, 2, 0)[ok] - out[ok][:, :3]).max() < 1e-4


def test_serving_config_requests_at_size():
    """The serving workload's largest requests on the 4.19M-surfel map: BEV
    2048^2 (RGB, SEM, ELEV at 0.05 m/px) and 1920x1080 perspective views.
    Each result is the same alone (plain server) and in a batched mix, bit for
    bit, and matches the FP64 oracle on sampled pixels."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render, rogs, serve
    m, field = scenes.grid_road_map(C=19)
    st = render.SurfelTensors.from_map(m)
    ex_np = np.zeros((1, 2), np.float32)
    ex = torch.as_tensor(ex_np, device="cuda")
    pool = scenes.serve_requests(field, n=400, seed=2)
    bev = [r for r in pool if r[0].kind == scenes.ORTHO and r[0].width == 2048]
    big = [next(r for r in bev if r[1] == ch) for ch in (1, 2, 4)]          # RGB, SEM, ELEV
    big += [r for r in pool if r[0].kind == scenes.PERSP and r[0].width == 1920][:2]
    assert len(big) == 5
    others = [r for r in pool if r[0].width <= 640][:12]
    cfg = rogs.rogs_default_config(19, 1 << 20, 1 << 22)
    kw = dict(memory_budget=8 << 30, record_capacity=4_000_000, pair_capacity=24_000_000)
    plain = serve.Server(cfg, st, ex, max_batch_views=1, max_inflight=1, **kw)
    try:
        alone = [plain.wait(plain.submit(c, ch), timeout=120.0) for c, ch in big]
    finally:
        plain.close()
    batched = serve.Server(cfg, st, ex, max_batch_views=16, max_inflight=3, **kw)
    try:
        mix = big + others
        order = np.random.default_rng(1).permutation(len(mix))
        tickets = {int(i): batched.submit(*mix[i]) for i in order}
        res = {i: batched.wait(t, timeout=120.0) for i, t in tickets.items()}
        assert batched.stats().failed == 0
    finally:
        batched.close()
    for i in range(len(big)):
        for k in alone[i]:
            np.testing.assert_array_equal(res[i][k], alone[i][k])
    rng = np.random.default_rng(3)
    for (cam, ch), r in zip(big, alone):
        H, W = cam.height, cam.width
        n = 300
        pix = np.stack([np.zeros(n, np.int32), rng.integers(0, W, n), rng.integers(H // 3 if cam.kind == scenes.PERSP else 0, H, n)],
                       -1).astype(np.int32)
        ref = oracle.render(m, [cam], ex_np, pix)
        ok = ref.amb == 0
        u, y = pix[:, 1], pix[:, 2]
        if ch & 1:
            assert np.abs(r["rgb"][:, y, u].T[ok] - ref.out[ok, :3]).max() < 1e-4
        if ch & 2:
            logits = ref.out[:, 3:3 + 19]
            top2 = np.sort(logits, -1)[:, -2:]
            clear = ok & (top2[:, 1] - top2[:, 0] > 1e-4)
            np.testing.assert_array_equal(r["sem"][y, u][clear], logits.argmax(-1)[clear])
        if ch & 4:
            cov = 1.0 - ref.T
            cam_z = -(cam.R.astype(np.float64).T @ cam.t.astype(np.float64))[2]
            D = ref.out[:, 3 + 19]
            with np.errstate(divide="ignore", invalid="ignore"):
                exp = np.where(cov >= 0.5, (cam_z - D / cov) if cam.kind == scenes.ORTHO else D / cov, np.nan)
            sure = ok & (np.abs(cov - 0.5) > 1e-4)
            got = r["elev"][y, u]
            assert np.array_equal(np.isnan(got[sure]), np.isnan(exp[sure]))
            fin = sure & ~np.isnan(exp)
            assert np.abs(got[fin] - exp[fin]).max() < 1e-3
        assert ok.mean() > 0.99
