"""ctypes binding of librogs (include/rogs.h), same names as the C-ABI.

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of librogs.so.  Importing this module loads the in-tree library and
raises if it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librogs.so")

ROGS_OK, ROGS_ERR_INVALID, ROGS_ERR_CAPACITY, ROGS_ERR_OOM = 0, 1, 2, 3
ROGS_ERR_CUDA, ROGS_ERR_TIMEOUT, ROGS_ERR_BUSY, ROGS_ERR_NOT_READY = 4, 5, 6, 7
ROGS_PERSP, ROGS_ORTHO = 0, 1
ROGS_MAX_VIEWS = 128
ROGS_MAX_CLASSES = 54

STATUS_NAMES = {0: "ROGS_OK", 1: "ROGS_ERR_INVALID", 2: "ROGS_ERR_CAPACITY", 3: "ROGS_ERR_OOM",
                4: "ROGS_ERR_CUDA", 5: "ROGS_ERR_TIMEOUT", 6: "ROGS_ERR_BUSY", 7: "ROGS_ERR_NOT_READY"}


class RogsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class rogs_config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("num_classes", C.c_int32),
                ("t_min", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("eps_dilate", C.c_float), ("near_plane", C.c_float), ("box_half_x", C.c_float),
                ("box_depth", C.c_float), ("jac_clamp", C.c_float), ("sort_tile", C.c_int32),
                ("record_capacity", C.c_int64), ("pair_capacity", C.c_int64)]


class rogs_camera(C.Structure):
    _fields_ = [("kind", C.c_int32), ("width", C.c_int32), ("height", C.c_int32), ("exposure_idx", C.c_int32),
                ("use_box_cull", C.c_int32), ("reserved", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R_wc", C.c_float * 9), ("t_wc", C.c_float * 3)]


class rogs_surfels(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("opacity", C.c_void_p),
                ("rgb", C.c_void_p), ("sem", C.c_void_p), ("n", C.c_int64), ("grid_index", C.c_void_p),
                ("grid_w", C.c_int32), ("grid_h", C.c_int32)]


class rogs_adam_group(C.Structure):
    _fields_ = [("param", C.c_void_p), ("grad", C.c_void_p), ("m", C.c_void_p), ("v", C.c_void_p),
                ("n", C.c_int64), ("stride", C.c_int32), ("lr", C.c_float), ("lr_end", C.c_float),
                ("decay_steps", C.c_int32), ("zero_lead", C.c_int32)]


ROGS_MAX_ADAM_GROUPS = 16


class rogs_grads(C.Structure):
    _fields_ = [("xyz", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p), ("opacity", C.c_void_p),
                ("rgb", C.c_void_p), ("sem", C.c_void_p), ("exposure", C.c_void_p)]


class rogs_counts(C.Structure):
    _fields_ = [("n_records", C.c_uint64), ("n_pairs", C.c_uint64), ("need_records", C.c_uint64),
                ("need_pairs", C.c_uint64), ("composited", C.c_uint64), ("status", C.c_uint32),
                ("n_views", C.c_uint32)]


class rogs_state_layout(C.Structure):
    _fields_ = [("header", C.c_uint64), ("records", C.c_uint64), ("rects", C.c_uint64), ("pair_rec", C.c_uint64),
                ("tile_range", C.c_uint64), ("pix_T", C.c_uint64), ("pix_last", C.c_uint64),
                ("views", C.c_uint64), ("tile_order", C.c_uint64), ("rec_feat", C.c_uint64),
                ("pair_mc", C.c_uint64), ("pair_blk", C.c_uint64),
                ("total_bytes", C.c_uint64),
                ("total_tiles", C.c_int64),
                ("total_pixels", C.c_int64)]


class rogs_serve_config(C.Structure):
    _fields_ = [("max_batch_views", C.c_int32), ("max_inflight", C.c_int32), ("max_queue", C.c_int32),
                ("reserved", C.c_int32), ("memory_budget", C.c_uint64), ("record_capacity", C.c_int64),
                ("pair_capacity", C.c_int64), ("timeout_s", C.c_double)]


class rogs_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("batches", C.c_uint64), ("views_rendered", C.c_uint64), ("pixels_rendered", C.c_uint64),
                ("pending", C.c_uint32), ("inflight", C.c_uint32)]


ROGS_CH_RGB, ROGS_CH_SEM, ROGS_CH_ELEV = 1, 2, 4


class rogs_profile(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("calls", C.c_uint64 * 8)]


STAGES = ("cull_project", "depth_sort", "pair_emit", "tile_sort", "composite_fwd", "loss", "composite_bwd",
          "project_bwd")

_lib = None


def lib():
    """The loaded librogs (raises if the extension was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"librogs.so not built at {LIB_PATH}; run __graft_entry__.build() "
                               "(python -m paper_2405_14342_gb300.build)")
        L = C.CDLL(LIB_PATH)
        P, S = C.c_void_p, C.c_int
        L.rogs_default_config.argtypes = [C.c_int32, C.c_int64, C.c_int64, C.POINTER(rogs_config)]
        L.rogs_create.argtypes = [C.POINTER(rogs_config), C.POINTER(P)]
        L.rogs_destroy.argtypes = [P]
        L.rogs_destroy.restype = None
        L.rogs_last_error.argtypes = [P]
        L.rogs_last_error.restype = C.c_char_p
        L.rogs_reserve.argtypes = [P, C.c_int64, C.POINTER(rogs_camera), C.c_int32, C.c_int32]
        L.rogs_state_layout_of.argtypes = [P, C.POINTER(rogs_camera), C.c_int32, C.POINTER(rogs_state_layout),
                                           C.POINTER(C.c_uint64)]
        L.rogs_state_counts.argtypes = [P, P, C.POINTER(rogs_counts), P]
        L.rogs_init_from_poses.argtypes = [P, P, C.c_int64, P, C.c_int64, C.c_int32, P, P, P, P]
        L.rogs_render_fwd.argtypes = [P, C.POINTER(rogs_surfels), C.POINTER(rogs_camera), C.c_int32, P, C.c_int32,
                                      P, P, P]
        L.rogs_loss.argtypes = [P, C.POINTER(rogs_camera), C.c_int32, P, P, P, P, C.c_float, C.c_float, P, P, P]
        L.rogs_render_bwd.argtypes = [P, C.POINTER(rogs_surfels), C.POINTER(rogs_camera), C.c_int32, P, C.c_int32,
                                      P, P, C.POINTER(rogs_grads), P]
        L.rogs_sort_pairs.argtypes = [P, P, P, C.c_int64, C.c_int32, P, P, P]
        L.rogs_train_graph_create.argtypes = [P, C.POINTER(rogs_surfels), C.POINTER(rogs_camera), C.c_int32, P,
                                              C.c_int32, P, P, P, P, P, C.c_float, C.c_float, C.c_float, P,
                                              C.POINTER(rogs_grads), P, C.POINTER(P)]
        L.rogs_smooth_loss.argtypes = [P, C.POINTER(rogs_surfels), C.c_float, P, P, P]
        L.rogs_elev_targets.argtypes = [P, C.POINTER(rogs_surfels), P, C.c_int64, C.c_float, P, P]
        L.rogs_elev_loss.argtypes = [P, C.POINTER(rogs_surfels), P, C.c_float, P, P, P]
        L.rogs_bev_export.argtypes = [P, C.POINTER(rogs_surfels), P, C.c_int32, C.c_int32, C.c_double, C.c_double,
                                      C.c_float, C.c_float, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P, P]
        L.rogs_adam_step.argtypes = [P, C.POINTER(rogs_adam_group), C.c_int32, C.c_int32, C.c_float, C.c_float,
                                     C.c_float, C.c_int32, P]
        L.rogs_train_step.argtypes = [P, C.POINTER(rogs_surfels), C.POINTER(rogs_camera), C.c_int32, P, C.c_int32,
                                      P, P, P, P, P, C.c_float, C.c_float, C.c_float, P, C.POINTER(rogs_grads), P]
        L.rogs_render_graph_create.argtypes = [P, C.POINTER(rogs_surfels), C.POINTER(rogs_camera), C.c_int32, P,
                                               C.c_int32, P, P, P, C.POINTER(P)]
        for base in ("rogs_loss", "rogs_train_step", "rogs_train_graph_create"):   # 8-bit target forms
            getattr(L, base + "_u8").argtypes = getattr(L, base).argtypes
        L.rogs_graph_launch.argtypes = [P, P]
        L.rogs_graph_destroy.argtypes = [P]
        L.rogs_graph_destroy.restype = None
        L.rogs_serve_result_bytes.argtypes = [C.POINTER(rogs_camera), C.c_int32, C.c_int32, C.POINTER(C.c_uint64)]
        L.rogs_serve_open.argtypes = [C.POINTER(rogs_config), C.POINTER(rogs_surfels), P, C.c_int32,
                                      C.POINTER(rogs_serve_config), C.POINTER(P)]
        L.rogs_serve_submit.argtypes = [P, C.POINTER(rogs_camera), C.c_int32, C.POINTER(C.c_uint64)]
        L.rogs_serve_poll.argtypes = [P, C.c_uint64, P, C.POINTER(C.c_int32)]
        L.rogs_serve_get_stats.argtypes = [P, C.POINTER(rogs_serve_stats)]
        L.rogs_serve_set_timeout.argtypes = [P, C.c_double]
        L.rogs_debug_fail_alloc.argtypes = [C.c_int32]
        L.rogs_bounds_checked.argtypes = [C.POINTER(C.c_uint32)]
        L.rogs_bounds_checked.restype = C.c_int32
        L.rogs_debug_fail_alloc.restype = None
        L.rogs_serve_close.argtypes = [P]
        L.rogs_serve_close.restype = None
        L.rogs_profile_enable.argtypes = [P, C.c_int32]
        L.rogs_profile_read.argtypes = [P, C.POINTER(rogs_profile)]
        L.rogs_measure_fp32_peak.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32), P]
        L.rogs_launch_count.argtypes = []
        L.rogs_launch_count.restype = C.c_uint64
        for name in ("rogs_train_step", "rogs_smooth_loss", "rogs_adam_step", "rogs_elev_targets", "rogs_elev_loss", "rogs_bev_export",
                     "rogs_serve_result_bytes", "rogs_serve_open", "rogs_serve_submit", "rogs_serve_poll",
                     "rogs_serve_get_stats", "rogs_serve_set_timeout", "rogs_measure_fp32_peak", "rogs_train_graph_create", "rogs_render_graph_create", "rogs_graph_launch",
                     "rogs_profile_enable", "rogs_profile_read","rogs_default_config", "rogs_create", "rogs_reserve", "rogs_state_layout_of",
                     "rogs_state_counts", "rogs_init_from_poses", "rogs_render_fwd", "rogs_loss",
                     "rogs_render_bwd", "rogs_sort_pairs", "rogs_loss_u8", "rogs_train_step_u8",
                     "rogs_train_graph_create_u8"):
            getattr(L, name).restype = S
        _lib = L
    return _lib


def _check(ctx, st):
    if st != ROGS_OK:
        msg = lib().rogs_last_error(ctx).decode() if ctx else ""
        raise RogsError(st, msg)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _target_entry(name, tgt_rgb, label):
    """The C entry for the targets' format: FP32 colour planes with int32
    labels (`name`), or 8-bit colour planes and labels (`name`_u8)."""
    import torch
    if tgt_rgb.dtype == torch.uint8:
        if label is not None and label.dtype != torch.uint8:
            raise TypeError("8-bit colour targets take uint8 labels")
        return getattr(lib(), name + "_u8")
    if tgt_rgb.dtype != torch.float32 or (label is not None and label.dtype != torch.int32):
        raise TypeError("targets are float32 colour with int32 labels, or uint8 colour with uint8 labels")
    return getattr(lib(), name)


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def cameras(cams) -> "C.Array":
    """Build a rogs_camera array from objects with kind/width/height/fx/fy/cx/cy/R/t/
    exposure_idx/use_box_cull attributes (e.g. scenes.Camera)."""
    arr = (rogs_camera * len(cams))()
    for i, c in enumerate(cams):
        a = arr[i]
        a.kind, a.width, a.height = int(c.kind), int(c.width), int(c.height)
        a.exposure_idx, a.use_box_cull, a.reserved = int(c.exposure_idx), int(c.use_box_cull), 0
        a.fx, a.fy, a.cx, a.cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        R = np.asarray(c.R, dtype=np.float32).ravel()
        t = np.asarray(c.t, dtype=np.float32).ravel()
        for k in range(9):
            a.R_wc[k] = float(R[k])
        for k in range(3):
            a.t_wc[k] = float(t[k])
    return arr


def surfels(xyz, scale, quat, opacity, rgb, sem, grid_index=None) -> rogs_surfels:
    s = rogs_surfels()
    s.xyz, s.scale, s.quat, s.opacity = xyz.data_ptr(), scale.data_ptr(), quat.data_ptr(), opacity.data_ptr()
    s.rgb, s.sem = rgb.data_ptr(), (sem.data_ptr() if sem is not None and sem.numel() else None)
    s.n = int(xyz.shape[0])
    if grid_index is not None:
        s.grid_index = grid_index.data_ptr()
        s.grid_h, s.grid_w = int(grid_index.shape[0]), int(grid_index.shape[1])
    return s


# ----------------------------------------------------------------- calls

def rogs_default_config(num_classes, record_capacity, pair_capacity, **over) -> rogs_config:
    cfg = rogs_config()
    _check(None, lib().rogs_default_config(num_classes, record_capacity, pair_capacity, C.byref(cfg)))
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def rogs_create(cfg: rogs_config):
    h = C.c_void_p()
    st = lib().rogs_create(C.byref(cfg), C.byref(h))
    if st != ROGS_OK:
        raise RogsError(st, "rogs_create failed")
    return h


def rogs_destroy(ctx):
    lib().rogs_destroy(ctx)


def rogs_last_error(ctx) -> str:
    return lib().rogs_last_error(ctx).decode()


def rogs_reserve(ctx, n_surfels, n_views, cam_arr=None, training=False):
    _check(ctx, lib().rogs_reserve(ctx, int(n_surfels), cam_arr, int(n_views), 1 if training else 0))


def rogs_measure_fp32_peak(reps=5, stream=None):
    """(measured FP32 FMA TFLOP/s, SM count) of the current device."""
    t, n = C.c_double(), C.c_int32()
    _check(None, lib().rogs_measure_fp32_peak(int(reps), C.byref(t), C.byref(n), _stream(stream)))
    return float(t.value), int(n.value)


def rogs_bounds_checked():
    """(True if the loaded library is the bounds-checked build, first failure code
    since the last call or 0)."""
    code = C.c_uint32()
    chk = lib().rogs_bounds_checked(C.byref(code))
    return bool(chk), int(code.value)


def rogs_debug_fail_alloc(fail_all: bool):
    lib().rogs_debug_fail_alloc(1 if fail_all else 0)


def rogs_state_layout_of(ctx, cam_arr, n_views):
    L = rogs_state_layout()
    elems = C.c_uint64()
    _check(ctx, lib().rogs_state_layout_of(ctx, cam_arr, n_views, C.byref(L), C.byref(elems)))
    return L, int(elems.value)


def rogs_state_counts(ctx, state, stream=None, check=True) -> rogs_counts:
    c = rogs_counts()
    st = lib().rogs_state_counts(ctx, _ptr(state), C.byref(c), _stream(stream))
    if check:
        _check(ctx, st)
    return c


def rogs_init_from_poses(ctx, grid_xy, poses_host: np.ndarray, exact_plane, out_z, out_quat, out_nearest=None,
                         stream=None):
    poses_host = np.ascontiguousarray(poses_host, dtype=np.float32).reshape(-1, 12)
    _check(ctx, lib().rogs_init_from_poses(ctx, _ptr(grid_xy), int(grid_xy.shape[0]),
                                           poses_host.ctypes.data_as(C.c_void_p), int(poses_host.shape[0]),
                                           int(bool(exact_plane)), _ptr(out_z), _ptr(out_quat), _ptr(out_nearest),
                                           _stream(stream)))


def rogs_render_fwd(ctx, surf: rogs_surfels, cam_arr, n_views, exposure_ab, out, state, stream=None):
    _check(ctx, lib().rogs_render_fwd(ctx, C.byref(surf), cam_arr, n_views, _ptr(exposure_ab),
                                      int(exposure_ab.shape[0]), _ptr(out), _ptr(state), _stream(stream)))


def rogs_loss(ctx, cam_arr, n_views, out, tgt_rgb, label, mask, lambda_c, lambda_s, loss, grad_out, stream=None):
    _check(ctx, _target_entry("rogs_loss", tgt_rgb, label)(ctx, cam_arr, n_views, _ptr(out), _ptr(tgt_rgb), _ptr(label), _ptr(mask),
                                float(lambda_c), float(lambda_s), _ptr(loss), _ptr(grad_out), _stream(stream)))


def rogs_render_bwd(ctx, surf: rogs_surfels, cam_arr, n_views, exposure_ab, state, grad_out, grads: rogs_grads,
                    stream=None):
    _check(ctx, lib().rogs_render_bwd(ctx, C.byref(surf), cam_arr, n_views, _ptr(exposure_ab),
                                      int(exposure_ab.shape[0]), _ptr(state), _ptr(grad_out), C.byref(grads),
                                      _stream(stream)))


def rogs_smooth_loss(ctx, surf: rogs_surfels, lambda_smooth, loss, grad_xyz=None, stream=None):
    _check(ctx, lib().rogs_smooth_loss(ctx, C.byref(surf), float(lambda_smooth), _ptr(loss), _ptr(grad_xyz),
                                       _stream(stream)))


def rogs_elev_targets(ctx, surf: rogs_surfels, points, radius, z_target, stream=None):
    _check(ctx, lib().rogs_elev_targets(ctx, C.byref(surf), _ptr(points), int(points.shape[0]), float(radius),
                                        _ptr(z_target), _stream(stream)))


def rogs_elev_loss(ctx, surf: rogs_surfels, z_target, lambda_z, loss, grad_xyz=None, stream=None):
    _check(ctx, lib().rogs_elev_loss(ctx, C.byref(surf), _ptr(z_target), float(lambda_z), _ptr(loss), _ptr(grad_xyz),
                                     _stream(stream)))


def rogs_bev_export(ctx, surf: rogs_surfels, exposure_ab, exposure_idx, x0, y1, res, cam_z, width, height, chunk,
                    batch, image, stream=None):
    _check(ctx, lib().rogs_bev_export(ctx, C.byref(surf), _ptr(exposure_ab), int(exposure_ab.shape[0]),
                                      int(exposure_idx), float(x0), float(y1), float(res), float(cam_z), int(width),
                                      int(height), int(chunk), int(batch), _ptr(image), _stream(stream)))


def rogs_adam_step(ctx, groups, step, beta1=0.9, beta2=0.999, eps=1e-8, zero_grad=True, stream=None):
    """groups: list of (param, grad, m, v, n, stride, lr) or (param, grad, m, v,
    n, stride, lr, lr_end, decay_steps, zero_lead) with device tensors (param /
    grad may be views offset into a larger tensor)."""
    arr = (rogs_adam_group * len(groups))()
    for i, grp in enumerate(groups):
        p, g, m, v, n, stride, lr = grp[:7]
        lr_end, decay, lead = grp[7:10] if len(grp) > 7 else (lr, 0, 0)
        arr[i].param, arr[i].grad = p.data_ptr(), g.data_ptr()
        arr[i].m, arr[i].v = m.data_ptr(), v.data_ptr()
        arr[i].n, arr[i].stride, arr[i].lr = int(n), int(stride), float(lr)
        arr[i].lr_end, arr[i].decay_steps, arr[i].zero_lead = float(lr_end), int(decay), int(lead)
    _check(ctx, lib().rogs_adam_step(ctx, arr, len(groups), int(step), float(beta1), float(beta2), float(eps),
                                     1 if zero_grad else 0, _stream(stream)))


def rogs_sort_pairs(ctx, keys_in, vals_in, key_bits, keys_out, vals_out, stream=None):
    _check(ctx, lib().rogs_sort_pairs(ctx, _ptr(keys_in), _ptr(vals_in), int(keys_in.numel()), int(key_bits),
                                      _ptr(keys_out), _ptr(vals_out), _stream(stream)))


def rogs_profile_enable(ctx, enable=True):
    _check(ctx, lib().rogs_profile_enable(ctx, int(bool(enable))))


def rogs_profile_read(ctx) -> dict:
    p = rogs_profile()
    _check(ctx, lib().rogs_profile_read(ctx, C.byref(p)))
    return {name: (float(p.ms[i]), int(p.calls[i])) for i, name in enumerate(STAGES)}


def rogs_launch_count() -> int:
    return int(lib().rogs_launch_count())


def rogs_train_graph_create(ctx, surf, cam_arr, n_views, exposure_ab, out, state, tgt_rgb, label, mask, lambda_c,
                            lambda_s, loss, grads: rogs_grads, stream=None, lambda_smooth=0.0):
    g = C.c_void_p()
    _check(ctx, _target_entry("rogs_train_graph_create", tgt_rgb, label)(ctx, C.byref(surf), cam_arr, n_views, _ptr(exposure_ab),
                                              int(exposure_ab.shape[0]), _ptr(out), _ptr(state), _ptr(tgt_rgb),
                                              _ptr(label), _ptr(mask), float(lambda_c), float(lambda_s),
                                              float(lambda_smooth), _ptr(loss),
                                              C.byref(grads), _stream(stream), C.byref(g)))
    return g


def rogs_train_step(ctx, surf, cam_arr, n_views, exposure_ab, out, state, tgt_rgb, label, mask, lambda_c, lambda_s,
                    loss, grads: rogs_grads, stream=None, lambda_smooth=0.0):
    _check(ctx, _target_entry("rogs_train_step", tgt_rgb, label)(ctx, C.byref(surf), cam_arr, n_views, _ptr(exposure_ab),
                                      int(exposure_ab.shape[0]), _ptr(out), _ptr(state), _ptr(tgt_rgb), _ptr(label),
                                      _ptr(mask), float(lambda_c), float(lambda_s), float(lambda_smooth), _ptr(loss),
                                      C.byref(grads),
                                      _stream(stream)))


def rogs_render_graph_create(ctx, surf, cam_arr, n_views, exposure_ab, out, state, stream=None):
    g = C.c_void_p()
    _check(ctx, lib().rogs_render_graph_create(ctx, C.byref(surf), cam_arr, n_views, _ptr(exposure_ab),
                                               int(exposure_ab.shape[0]), _ptr(out), _ptr(state), _stream(stream),
                                               C.byref(g)))
    return g


def rogs_graph_launch(graph, stream=None):
    _check(None, lib().rogs_graph_launch(graph, _stream(stream)))


def rogs_graph_destroy(graph):
    lib().rogs_graph_destroy(graph)


def rogs_serve_result_bytes(cam_arr, channels, num_classes) -> int:
    b = C.c_uint64()
    _check(None, lib().rogs_serve_result_bytes(cam_arr, int(channels), int(num_classes), C.byref(b)))
    return int(b.value)


def rogs_serve_open(cfg_render: rogs_config, surf: rogs_surfels, exposure_ab, cfg: rogs_serve_config):
    h = C.c_void_p()
    _check(None, lib().rogs_serve_open(C.byref(cfg_render), C.byref(surf), _ptr(exposure_ab),
                                       int(exposure_ab.shape[0]), C.byref(cfg), C.byref(h)))
    return h


def rogs_serve_submit(srv, cam_arr, channels) -> int:
    """Returns the ticket; raises RogsError (ROGS_ERR_BUSY / _OOM / _INVALID)."""
    t = C.c_uint64()
    _check(None, lib().rogs_serve_submit(srv, cam_arr, int(channels), C.byref(t)))
    return int(t.value)


def rogs_serve_poll(srv, ticket, host_buf) -> bool:
    """True when finished (result copied into host_buf), False while not ready."""
    d = C.c_int32()
    st = lib().rogs_serve_poll(srv, C.c_uint64(ticket), host_buf, C.byref(d))
    if st == ROGS_ERR_NOT_READY:
        return False
    _check(None, st)
    return bool(d.value)


def rogs_serve_get_stats(srv) -> rogs_serve_stats:
    s = rogs_serve_stats()
    _check(None, lib().rogs_serve_get_stats(srv, C.byref(s)))
    return s


def rogs_serve_set_timeout(srv, timeout_s):
    _check(None, lib().rogs_serve_set_timeout(srv, float(timeout_s)))


def rogs_serve_close(srv):
    lib().rogs_serve_close(srv)
