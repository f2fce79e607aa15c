"""Chunked BEV export (rogs_bev_export): the stitched chunks against one
large orthographic render of the same rectangle (seams included) and against
the FP64 oracle."""
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


def test_chunked_export_equals_one_render(R):
    m = scenes.tiny_map(C=5)
    res, W, H, chunk, cam_z = 0.05, 128, 96, 48, 20.0
    x0, y1 = 0.1, 6.1
    ex_np = np.array([[0.05, 0.01]], np.float32)
    ex = torch.as_tensor(ex_np, device="cuda")
    rr = R.Renderer(5, record_capacity=1 << 16, pair_capacity=1 << 20)
    st = R.SurfelTensors.from_map(m)
    img = rr.bev_export(st, ex, x0, y1, res, W, H, chunk=chunk, batch=3, cam_z=cam_z).cpu().numpy()
    # one camera over the whole rectangle, same conventions
    cam = scenes.make_camera(scenes.ORTHO, W, H, 1 / res, 1 / res,
                             np.array([[1.0, 0, 0], [0, -1.0, 0], [0, 0, -1.0]]),
                             (x0 + 0.5 * W * res, y1 - 0.5 * H * res, cam_z))
    fr = rr.frame([cam])
    rr.forward(st, fr, ex)
    torch.cuda.synchronize()
    one = fr.view(0, 5).cpu().numpy()
    pix = oracle.full_pixels([cam])
    ref = oracle.render(m, [cam], ex_np, pix)
    ok = (ref.amb == 0).reshape(H, W)
    assert ok.mean() > 0.999
    diff = np.abs(img - one)
    assert diff[:8][:, ok].max() <= 1e-4                     # rgb and logits
    assert diff[8][ok].max() <= 1e-4 * cam_z                 # depth channel
    # the seams: the rows and columns where chunks meet
    for c in range(chunk, W, chunk):
        assert diff[:8, :, c - 1:c + 1][:, ok[:, c - 1:c + 1]].max() <= 1e-4
    for r in range(chunk, H, chunk):
        assert diff[:8, r - 1:r + 1, :][:, ok[r - 1:r + 1, :]].max() <= 1e-4
    out = ref.out.reshape(H, W, -1)
    assert np.abs(img[:3].transpose(1, 2, 0)[ok] - out[ok][:, :3]).max() <= 1e-4


def test_export_rejects_bad_arguments(R):
    from paper_2405_14342_gb300 import rogs
    m = scenes.tiny_map(C=2)
    rr = R.Renderer(2, record_capacity=1 << 14, pair_capacity=1 << 16)
    st = R.SurfelTensors.from_map(m)
    ex = torch.zeros(1, 2, device="cuda")
    with pytest.raises(rogs.RogsError) as ei:
        rr.bev_export(st, ex, 0.0, 6.0, 0.05, 64, 64, chunk=32, batch=0)
    assert ei.value.status == rogs.ROGS_ERR_INVALID
    with pytest.raises(rogs.RogsError):
        rr.bev_export(st, ex, 0.0, 6.0, 0.05, 64, 64, chunk=32, batch=2, exposure_idx=3)
