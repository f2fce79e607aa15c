"""The bounds-checked build (-DROGS_CHECKED: every index the kernels take
from device data is tested before use; compute-sanitizer is not available on
the GPU machines) runs the forward, the separate loss and backward, the fused
training step at the scene size, graph capture and replay, lists of 10,000
entries and a capacity overflow with no index out of range, and its results
are those of the normal build (the tests change no arithmetic: outputs and
losses bit-identical, gradients up to the order of their atomic sums)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2405_14342_gb300 import rogs
rogs.LIB_PATH = LIB
from paper_2405_14342_gb300 import render as R, scenes
torch.cuda.set_device(0)
res = {}

def run(name, C, m, cams, ex, cap=(1 << 18, 1 << 21), step=False, grid=None):
    rr = R.Renderer(C, record_capacity=cap[0], pair_capacity=cap[1])
    st = R.SurfelTensors.from_map(m, grid_index=grid)
    ext = torch.as_tensor(np.asarray(ex, np.float32), device="cuda")
    fr = rr.frame(cams)
    tg = scenes.random_targets(cams, C, seed=3)
    trgb, lab, msk = R.targets_to_device(tg)
    grads = R.zero_grads(st, ext)
    if step:
        loss = torch.empty(1, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            rr.train_step(st, fr, ext, trgb, lab, msk, loss, grads, lambda_smooth=0.003 if grid is not None else 0.0)
            g = rr.train_graph(st, fr, ext, trgb, lab, msk, loss, grads,
                               lambda_smooth=0.003 if grid is not None else 0.0, stream=s)
            g.launch(s)
        s.synchronize()
        g.close()
        res[name + "/loss"] = float(loss.item())
    else:
        rr.forward(st, fr, ext)
        l, gout = rr.loss(fr, trgb, lab, msk)
        rr.backward(st, fr, ext, gout, grads=grads)
        torch.cuda.synchronize()
        res[name + "/loss"] = float(l.item())
    cnt = rr.counts(fr, check=False)
    res[name + "/status"] = int(cnt.status)
    res[name + "/out"] = float(fr.out.double().abs().sum().item())
    for k, v in grads.items():
        res[name + "/g_" + k] = float(v.double().abs().sum().item())
    np.save(OUT + "_" + name + ".npy", fr.out.cpu().numpy())
    rr.close()

m = scenes.tiny_map(C=8)
cams = [scenes.tiny_camera(), scenes.bev_camera((3.0, 3.1), 72, res_m=0.08, height_m=15.0)]
run("tiny", 8, m, cams, [[0.05, -0.02]])
run("overflow", 8, m, cams, [[0.05, -0.02]], cap=(1 << 18, 5000))
n1 = 100
g = (np.arange(n1) * 0.012).astype(np.float32)
xx, yy = np.meshgrid(g, g)
n = n1 * n1
mm = scenes.SurfelMap(xyz=np.stack([xx.ravel(), yy.ravel(), np.zeros(n)], -1).astype(np.float32),
                      scale=np.full((n, 2), 0.3, np.float32), quat=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                      opacity=np.full(n, 0.05, np.float32), rgb=np.full((n, 3), 0.5, np.float32),
                      sem=np.zeros((n, 2), np.float32))
run("long_lists", 2, mm, [scenes.bev_camera((0.6, 0.6), 32, res_m=0.05, height_m=10.0)], [[0.0, 0.0]])
ms, field = scenes.strip_map(C=19)
run("scene", 19, ms, scenes.surround_rig(field, 8), scenes.exposure_params(6), cap=(2_000_000, 12_000_000), step=True,
    grid=scenes.grid_index(ms))
chk, code = rogs.rogs_bounds_checked()
res["checked"], res["code"] = chk, code
print("RESULT " + json.dumps(res))
"""


def _run(lib, out):
    code = "ROOT = %r\nLIB = %r\nOUT = %r\n" % (ROOT, lib, out) + SCRIPT
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    line = [l for l in p.stdout.splitlines() if l.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_checked_build_finds_no_bad_index_and_changes_nothing(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_14342_gb300 import build
    plain = build.build()
    checked = build.build(checked=True)
    a = _run(checked, str(tmp_path / "checked"))
    b = _run(plain, str(tmp_path / "plain"))
    assert a["checked"] is True and b["checked"] is False
    assert a["code"] == 0, a["code"]
    assert a["overflow/status"] != 0                    # the overflow case did overflow
    for k in b:
        if k in ("checked", "code"):
            continue
        if "/g_" in k:      # gradients are summed with atomics: equal up to the order of the additions
            assert abs(a[k] - b[k]) <= 1e-5 * abs(b[k]), (k, a[k], b[k])
        else:
            assert a[k] == b[k], (k, a[k], b[k])
    for name in ("tiny", "overflow", "long_lists", "scene"):
        np.testing.assert_array_equal(np.load(tmp_path / f"checked_{name}.npy"), np.load(tmp_path / f"plain_{name}.npy"))
