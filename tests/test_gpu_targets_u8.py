"""8-bit targets (rogs_loss_u8, rogs_train_step_u8, rogs_train_graph_create_u8):
the colour target is value / 255 rounded to the nearest float and the label a
class id, so every result equals the FP32 / int32 form given those values
(Sec. 3.3.2, Eqs. 8, 9).  The FP32 form is checked against the FP64 oracle in
test_gpu_parity.py and test_gpu_scale.py."""
import numpy as np
import pytest

from paper_2405_14342_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from _util import normwise  # noqa: E402


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import render
    return render


def _u8_targets(cams, C, seed):
    """Random 8-bit targets in the output pixel order (colour planes per view,
    labels with some 255 = no label, mask) and the same values as FP32 / int32."""
    g = np.random.default_rng(seed)
    rgb8, lab8, msk = [], [], []
    for c in cams:
        n = c.width * c.height
        rgb8.append(g.integers(0, 256, size=3 * n, dtype=np.uint8))
        lb = g.integers(0, C, size=n).astype(np.uint8) if C > 0 else np.full(n, 255, np.uint8)
        lb[g.uniform(size=n) < 0.05] = 255
        lab8.append(lb)
        msk.append((g.uniform(size=n) < 0.8).astype(np.uint8))
    rgb8, lab8, msk = np.concatenate(rgb8), np.concatenate(lab8), np.concatenate(msk)
    rgb32 = rgb8.astype(np.float32) / np.float32(255.0)   # IEEE division, rounded to nearest
    dev = lambda a: torch.as_tensor(a, device="cuda").contiguous()  # noqa: E731
    return (dev(rgb8), dev(lab8), dev(msk)), (dev(rgb32), dev(lab8.astype(np.int32)), dev(msk))


def test_u8_colour_is_value_over_255_for_every_value(R):
    """An output equal to k / 255 (IEEE) against the 8-bit target k leaves no
    L1 residue for any of the 256 values: loss exactly 0, zero colour gradient."""
    m = scenes.tiny_map(C=3)
    cams = [scenes.tiny_camera()]
    rr = R.Renderer(3, record_capacity=1 << 16, pair_capacity=1 << 20)
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame(cams)
    ex = torch.zeros((1, 2), device="cuda")
    rr.forward(st, fr, ex)
    n = cams[0].width * cams[0].height
    k = (np.arange(3 * n) * 7 + 3) % 256                      # every value, in every plane
    rgb8 = torch.as_tensor(k.astype(np.uint8), device="cuda")
    fr.out[:3 * n] = torch.as_tensor(k.astype(np.float32) / np.float32(255.0), device="cuda")
    lab8 = torch.zeros(n, dtype=torch.uint8, device="cuda")
    msk = torch.ones(n, dtype=torch.uint8, device="cuda")
    loss, gout = rr.loss(fr, rgb8, lab8, msk, lambda_c=1.0, lambda_s=0.0)
    torch.cuda.synchronize()
    assert loss.item() == 0.0
    assert torch.count_nonzero(gout[:3 * n]).item() == 0
    # targets one step off: a positive loss (the check above is not vacuous)
    rgb8b = torch.as_tensor(((k + 1) % 256).astype(np.uint8), device="cuda")
    loss_b, _ = rr.loss(fr, rgb8b, lab8, msk, lambda_c=1.0, lambda_s=0.0)
    torch.cuda.synchronize()
    assert loss_b.item() > 0.0


def test_loss_u8_equals_fp32_targets_bit_for_bit(R):
    m = scenes.tiny_map(C=8)
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 96, res_m=0.06, height_m=20.0)]
    rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame(cams)
    rr.forward(st, fr, torch.zeros((1, 2), device="cuda"))
    t8, t32 = _u8_targets(cams, 8, seed=11)
    l8, g8 = rr.loss(fr, *t8)
    l32, g32 = rr.loss(fr, *t32)
    torch.cuda.synchronize()
    assert l8.item() == l32.item() and l8.item() > 0.0
    assert torch.equal(g8, g32)


def test_train_step_and_graph_u8_equal_fp32_targets(R):
    m = scenes.tiny_map(C=8)
    cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.0), 96, res_m=0.06, height_m=20.0)]
    ex = torch.as_tensor(np.array([[0.05, 0.01]], np.float32), device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rr = R.Renderer(8, record_capacity=1 << 16, pair_capacity=1 << 20)
        st = R.SurfelTensors.from_map(m)
        t8, t32 = _u8_targets(cams, 8, seed=12)
        res = {}
        for name, tg in (("f32", t32), ("u8", t8)):
            fr = rr.frame(cams)
            loss = torch.empty(1, device="cuda")
            grads = R.zero_grads(st, ex)
            rr.train_step(st, fr, ex, *tg, loss, grads)
            res[name] = (fr, loss, grads)
        fr_g = rr.frame(cams)
        loss_g = torch.empty(1, device="cuda")
        grads_g = R.zero_grads(st, ex)
        graph = rr.train_graph(st, fr_g, ex, *t8, loss_g, grads_g)
        graph.launch()
        s.synchronize()
        (fa, la, ga), (fb, lb, gb) = res["f32"], res["u8"]
        assert torch.equal(fa.out, fb.out) and torch.equal(fr_g.out, fa.out)
        # per-pixel loss terms are identical and summed in a fixed order
        assert la.item() == lb.item() == loss_g.item() and la.item() > 0.0
        for key in ga:   # gradients: the same terms, atomics in any order
            assert normwise(gb[key].cpu().numpy(), ga[key].cpu().numpy()) < 1e-5, key
            assert normwise(grads_g[key].cpu().numpy(), ga[key].cpu().numpy()) < 1e-5, key
        graph.close()


def test_mixed_target_types_are_refused(R):
    m = scenes.tiny_map(C=4)
    cams = [scenes.tiny_camera()]
    rr = R.Renderer(4, record_capacity=1 << 16, pair_capacity=1 << 20)
    st = R.SurfelTensors.from_map(m)
    fr = rr.frame(cams)
    rr.forward(st, fr, torch.zeros((1, 2), device="cuda"))
    t8, t32 = _u8_targets(cams, 4, seed=13)
    with pytest.raises(TypeError):
        rr.loss(fr, t8[0], t32[1], t8[2])         # 8-bit colour with int32 labels
    with pytest.raises(TypeError):
        rr.loss(fr, t32[0], t8[1], t32[2])        # FP32 colour with 8-bit labels
    with pytest.raises(TypeError):
        rr.loss(fr, t32[0].double(), t32[1], t32[2])
