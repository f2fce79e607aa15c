"""Failure handling and the asynchronous contract, on the host side of the
C-ABI: simulated allocation failures come back as ROGS_ERR_OOM and leave the
library usable; after rogs_reserve the rendering calls allocate nothing (so
they also run while every allocation would fail); the first backward of a
fresh, unreserved context on a non-blocking stream clears its new gradient
rows on that stream before its kernels read them."""
import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _util import check_gradients, planar_grad_from_pixels  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render, rogs
    yield render
    rogs.rogs_debug_fail_alloc(False)


def _setup(C=8):
    m = scenes.tiny_map(C=C)
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 64, res_m=0.1, height_m=20.0)]
    tg = scenes.random_targets(cams, C, seed=3)
    return m, cams, tg


def test_allocation_failure_is_reported_and_recovers(R):
    from paper_2405_14342_gb300 import rogs, serve
    m, cams, tg = _setup()
    st = R.SurfelTensors.from_map(m)
    ex = torch.zeros(1, 2, device="cuda")
    rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)     # no reserve: scratch grows on use
    fr = rr.frame(cams)
    rogs.rogs_debug_fail_alloc(True)
    try:
        with pytest.raises(rogs.RogsError) as ei:
            R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
        assert ei.value.status == rogs.ROGS_ERR_OOM
        with pytest.raises(rogs.RogsError) as ei:
            rr.forward(st, fr, ex)                 # the visibility scratch cannot grow
        assert ei.value.status == rogs.ROGS_ERR_OOM
        with pytest.raises(rogs.RogsError) as ei:
            serve.Server(rogs.rogs_default_config(8, 1 << 16, 1 << 20), st, ex, max_inflight=1,
                         memory_budget=64 << 20, record_capacity=1 << 16, pair_capacity=1 << 20)
        assert ei.value.status == rogs.ROGS_ERR_OOM
    finally:
        rogs.rogs_debug_fail_alloc(False)
    rr.forward(st, fr, ex)                         # the same context works once memory is there
    torch.cuda.synchronize()
    pix = oracle.full_pixels(cams)
    ref = oracle.render(m, cams, np.zeros((1, 2)), pix)
    from _util import gpu_pixels
    got = gpu_pixels(fr, 8, pix)
    ok = ref.amb == 0
    assert np.abs(got[ok, :3] - ref.out[ok, :3]).max() < 1e-4


def test_reserved_context_allocates_nothing(R):
    """After rogs_reserve(training) for a camera set, forward, loss, backward,
    the fused training step and graph capture and replay run while every
    library allocation would fail."""
    from paper_2405_14342_gb300 import rogs
    m, cams, tg = _setup()
    st = R.SurfelTensors.from_map(m, grid_index=scenes.grid_index(m))
    ex = torch.zeros(1, 2, device="cuda")
    rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
    rr.reserve(st.n, cams=cams, training=True)
    fr = rr.frame(cams)
    trgb, lab, msk = R.targets_to_device(tg)
    grads = R.zero_grads(st, ex)
    loss = torch.empty(1, device="cuda")
    s = torch.cuda.Stream()
    rogs.rogs_debug_fail_alloc(True)
    try:
        with torch.cuda.stream(s):
            rr.forward(st, fr, ex)
            l2, gout = rr.loss(fr, trgb, lab, msk)
            rr.backward(st, fr, ex, gout, grads=grads)
            rr.train_step(st, fr, ex, trgb, lab, msk, loss, grads, lambda_smooth=0.003)
            g = rr.train_graph(st, fr, ex, trgb, lab, msk, loss, grads, lambda_smooth=0.003, stream=s)
            g.launch(s)
        s.synchronize()
    finally:
        rogs.rogs_debug_fail_alloc(False)
    g.close()
    assert torch.isfinite(loss).all() and grads["rgb"].abs().sum() > 0


def test_first_backward_of_a_fresh_context_on_a_nonblocking_stream(R):
    """No reserve: the backward's gradient rows are allocated and cleared by the
    first backward itself, on the caller's non-blocking stream, right before
    its kernels; the gradients still match the oracle."""
    m, cams, tg = _setup()
    ex = np.array([[0.04, -0.01]], np.float32)
    s = torch.cuda.Stream()          # torch creates it non-blocking with respect to the legacy stream
    with torch.cuda.stream(s):
        rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
        st = R.SurfelTensors.from_map(m)
        ext = torch.as_tensor(ex, device="cuda")
        fr = rr.frame(cams)
        pix = oracle.full_pixels(cams)
        ref = oracle.render(m, cams, ex, pix)
        rgb, lb, mk = oracle.gather_targets(tg, pix)
        mk = mk * (ref.amb == 0)
        L, gout = oracle.loss(ref.out, rgb, lb, mk, 8)
        gpl = torch.as_tensor(planar_grad_from_pixels(fr, 8, pix, gout), device="cuda")
        rr.forward(st, fr, ext)
        g = rr.backward(st, fr, ext, gpl)
    s.synchronize()
    gref = oracle.backward(m, cams, ex, pix, gout)
    check_gradients({k: v.cpu().numpy() for k, v in g.items()}, gref.as_dict())
