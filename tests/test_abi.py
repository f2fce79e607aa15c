"""The C-ABI library loads and exports every function declared in include/rogs.h
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rogs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:rogs_status|void|const char\*|u?int(?:32|64)_t|size_t)\s+(rogs_\w+)\s*\(",
                           src, flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rogs_create", "rogs_destroy", "rogs_init_from_poses", "rogs_render_fwd", "rogs_render_bwd",
              "rogs_loss", "rogs_state_counts", "rogs_sort_pairs", "rogs_launch_count", "rogs_train_step",
              "rogs_adam_step", "rogs_smooth_loss", "rogs_bev_export", "rogs_sort_pairs_noalloc"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2405_14342_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_2405_14342_gb300 import rogs
    monkeypatch.setattr(rogs, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(rogs, "_lib", None)
    with pytest.raises(RuntimeError):
        rogs.lib()


def test_default_config_without_gpu():
    from paper_2405_14342_gb300 import rogs
    cfg = rogs.rogs_default_config(19, 1000, 2000)
    assert cfg.tile_w == 16 and cfg.tile_h == 16 and cfg.num_classes == 19
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and abs(cfg.t_min - 1e-4) < 1e-11


def test_binding_picks_the_entry_point_by_target_format():
    """FP32 colour with int32 labels goes to the plain entry points, 8-bit
    colour with 8-bit labels to the _u8 ones; mixed or other types are refused
    before any call (no GPU needed: only the symbol is looked up)."""
    torch = pytest.importorskip("torch")
    from paper_2405_14342_gb300 import rogs
    L = rogs.lib()
    f32, i32, u8 = torch.zeros(3), torch.zeros(1, dtype=torch.int32), torch.zeros(3, dtype=torch.uint8)
    for name in ("rogs_loss", "rogs_train_step", "rogs_train_graph_create"):
        assert rogs._target_entry(name, f32, i32) is getattr(L, name)
        assert rogs._target_entry(name, u8, u8[:1]) is getattr(L, name + "_u8")
        assert rogs._target_entry(name, u8, None) is getattr(L, name + "_u8")   # no classes: no labels
        for rgb, lab in ((u8, i32), (f32, u8[:1]), (f32.double(), i32), (f32, i32.long())):
            with pytest.raises(TypeError):
                rogs._target_entry(name, rgb, lab)
