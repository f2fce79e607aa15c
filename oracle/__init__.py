"""FP64 CPU oracle for meshgrid-surfel splatting (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package.  It is independent of the CUDA path:
it shares no source, header or helper with ``paper_2405_14342_gb300``; both
take their inputs from the seeded generators in
``paper_2405_14342_gb300.scenes``, which hold none of the method's arithmetic.

Each wrapper below calls one function of ``rogs_oracle.c``; the equations it
follows are cited there (RoGs, Sec. 3.1-3.3, Eqs. 2, 4-9, S1-S2).  The
elevation smoothness loss is plain numpy in ``oracle/smooth.py``, the
optimiser step in ``oracle/adam.py`` and the LiDAR elevation loss in
``oracle/lidar.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rogs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None

# t_min, alpha_min, alpha_max, eps, near, box_half_x, box_depth, jac_clamp, lambda_c, lambda_s
DEFAULT_CFG = dict(t_min=1e-4, alpha_min=1.0 / 255.0, alpha_max=0.99, eps=0.3, near=0.2,
                   box_half_x=20.0, box_depth=40.0, jac_clamp=1.3, lambda_c=1.0, lambda_s=0.06)
_CFG_ORDER = ["t_min", "alpha_min", "alpha_max", "eps", "near", "box_half_x", "box_depth",
              "jac_clamp", "lambda_c", "lambda_s"]


def build(force: bool = False, src: str = _SRC, out: str = _LIB_PATH) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction)."""
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(src):
        return out
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def load(path: str = None):
    global _lib
    with _lock:
        if path is not None:
            return _bind(C.CDLL(path))
        if _lib is None:
            _lib = _bind(C.CDLL(build()))
        return _lib


class using:
    """Context manager: route every wrapper through another build of the
    oracle (the tests use it to show that a planted mistake fails a pin)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        load()
        self._saved = _lib
        _lib = _bind(C.CDLL(self.path))
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _bind(lib):
    P = C.c_void_p
    lib.orc_render.restype = None
    lib.orc_project.restype = None
    lib.orc_backward.restype = None
    lib.orc_loss.restype = C.c_double
    lib.orc_bin.restype = C.c_int64
    lib.orc_init_from_poses.restype = C.c_int
    lib.orc_num_threads.restype = C.c_int
    lib.orc_set_threads.argtypes = [C.c_int]
    return lib


def cfg_array(**over) -> np.ndarray:
    d = dict(DEFAULT_CFG)
    d.update(over)
    return np.array([d[k] for k in _CFG_ORDER], dtype=np.float32)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a if shape is None else a.reshape(shape)


def _cams(cams):
    ci = np.array([[c.kind, c.width, c.height, c.exposure_idx, c.use_box_cull] for c in cams], dtype=np.int32)
    cf = np.array([[c.fx, c.fy, c.cx, c.cy, *np.asarray(c.R, np.float32).ravel(), *np.asarray(c.t, np.float32)]
                   for c in cams], dtype=np.float32)
    return np.ascontiguousarray(ci), np.ascontiguousarray(cf)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _map(m):
    # float32 parameters widen exactly; float64 ones (finite differences) pass through
    return (_f64(m.xyz), _f64(m.scale), _f64(m.quat), _f64(m.opacity), _f64(m.rgb), _f64(m.sem))


def full_pixels(cams, views=None):
    """Pixel list (view, u, v) covering whole frames, view-major, row-major."""
    out = []
    for vi, c in enumerate(cams):
        if views is not None and vi not in views:
            continue
        vv, uu = np.meshgrid(np.arange(c.height), np.arange(c.width), indexing="ij")
        out.append(np.stack([np.full(uu.size, vi), uu.ravel(), vv.ravel()], -1))
    return np.ascontiguousarray(np.concatenate(out).astype(np.int32))


def crop_pixels(view, u0, v0, w, h):
    vv, uu = np.meshgrid(np.arange(v0, v0 + h), np.arange(u0, u0 + w), indexing="ij")
    return np.ascontiguousarray(np.stack([np.full(uu.size, view), uu.ravel(), vv.ravel()], -1).astype(np.int32))


class Render:
    def __init__(self, out, T, sumw, ncomp, last, amb, sig):
        self.out, self.T, self.sumw, self.ncomp, self.last, self.amb = out, T, sumw, ncomp, last, amb
        self.sig = sig


def render(m, cams, exposure, pix, cfg=None) -> Render:
    """Brute-force render of a pixel list: every surfel at every pixel (Eq. 6)."""
    lib = load()
    cfg = cfg_array() if cfg is None else cfg
    xyz, sc, q, op, rgb, sem = _map(m)
    ci, cf = _cams(cams)
    ex = _f64(exposure, (-1, 2))
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    n_pix = pix.shape[0]
    Cn = m.num_classes
    out = np.zeros((n_pix, 3 + Cn + 1), np.float64)
    T = np.zeros(n_pix); sw = np.zeros(n_pix)
    nc = np.zeros(n_pix, np.int64); last = np.zeros(n_pix, np.int64); amb = np.zeros(n_pix, np.int32)
    sig = np.zeros(n_pix, np.uint64)
    lib.orc_render(C.c_int64(m.n), C.c_int(Cn), _p(xyz), _p(sc), _p(q), _p(op), _p(rgb), _p(sem),
                   C.c_int(len(cams)), _p(ci), _p(cf), _p(ex), _p(cfg), C.c_int64(n_pix), _p(pix),
                   _p(out), _p(T), _p(sw), _p(nc), _p(last), _p(amb), _p(sig))
    return Render(out, T, sw, nc, last, amb, sig)


class Projection:
    def __init__(self, vis, mu, cov, con, depth, key):
        self.vis, self.mu, self.cov, self.con, self.depth, self.key = vis, mu, cov, con, depth, key


def project(m, cams, cfg=None) -> Projection:
    lib = load()
    cfg = cfg_array() if cfg is None else cfg
    xyz, sc, q, op, _, _ = _map(m)
    ci, cf = _cams(cams)
    V, n = len(cams), m.n
    vis = np.zeros((V, n), np.int8); mu = np.zeros((V, n, 2)); cov = np.zeros((V, n, 3))
    con = np.zeros((V, n, 3)); depth = np.zeros((V, n)); key = np.zeros((V, n), np.float32)
    lib.orc_project(C.c_int64(n), _p(xyz), _p(sc), _p(q), _p(op), C.c_int(V), _p(ci), _p(cf), _p(cfg),
                    _p(vis), _p(mu), _p(cov), _p(con), _p(depth), _p(key))
    return Projection(vis.astype(bool), mu, cov, con, depth, key)


def loss(out, tgt_rgb, label, mask, C_, cfg=None, grad=True):
    """Eqs. 8-9 over a pixel list; returns (L, dL/dout or None)."""
    lib = load()
    cfg = cfg_array() if cfg is None else cfg
    out = np.ascontiguousarray(out, dtype=np.float64)
    n_pix = out.shape[0]
    tr = _f32(tgt_rgb, (n_pix, 3))
    lb = np.ascontiguousarray(label, dtype=np.int32).reshape(n_pix)
    mk = np.ascontiguousarray(mask, dtype=np.uint8).reshape(n_pix)
    g = np.zeros_like(out) if grad else None
    L = lib.orc_loss(C.c_int64(n_pix), C.c_int(C_), _p(out), _p(tr), _p(lb), _p(mk), _p(cfg),
                     _p(g) if grad else None)
    return float(L), g


class Grads:
    def __init__(self, **kw):
        self.__dict__.update(kw)

    def as_dict(self):
        return dict(self.__dict__)


def backward(m, cams, exposure, pix, gout, cfg=None) -> Grads:
    lib = load()
    cfg = cfg_array() if cfg is None else cfg
    xyz, sc, q, op, rgb, sem = _map(m)
    ci, cf = _cams(cams)
    ex = _f64(exposure, (-1, 2))
    pix = np.ascontiguousarray(pix, dtype=np.int32)
    gout = np.ascontiguousarray(gout, dtype=np.float64)
    n, Cn = m.n, m.num_classes
    g = Grads(xyz=np.zeros((n, 3)), scale=np.zeros((n, 2)), quat=np.zeros((n, 4)), opacity=np.zeros(n),
              rgb=np.zeros((n, 3)), sem=np.zeros((n, Cn)), exposure=np.zeros((ex.shape[0], 2)))
    lib.orc_backward(C.c_int64(n), C.c_int(Cn), _p(xyz), _p(sc), _p(q), _p(op), _p(rgb), _p(sem),
                     C.c_int(len(cams)), _p(ci), _p(cf), _p(ex), C.c_int(ex.shape[0]), _p(cfg),
                     C.c_int64(pix.shape[0]), _p(pix), _p(gout),
                     _p(g.xyz), _p(g.scale), _p(g.quat), _p(g.opacity), _p(g.rgb), _p(g.sem), _p(g.exposure))
    return g


def gather_targets(targets, pix):
    """Per-pixel target rgb (n,3), label (n,), mask (n,) for a pixel list."""
    v, u, y = pix[:, 0], pix[:, 1], pix[:, 2]
    rgb = np.zeros((pix.shape[0], 3), np.float32)
    lab = np.zeros(pix.shape[0], np.int32)
    msk = np.zeros(pix.shape[0], np.uint8)
    for vi in np.unique(v):
        s = v == vi
        rgb[s] = targets.rgb[vi][:, y[s], u[s]].T
        lab[s] = targets.label[vi][y[s], u[s]]
        msk[s] = targets.mask[vi][y[s], u[s]]
    return rgb, lab, msk


def loss_and_grads(m, cams, exposure, targets, pix, cfg=None):
    """Forward, loss (Eqs. 8-9) and FP64 gradient for a pixel list."""
    r = render(m, cams, exposure, pix, cfg)
    rgb, lab, msk = gather_targets(targets, pix)
    L, gout = loss(r.out, rgb, lab, msk, m.num_classes, cfg)
    g = backward(m, cams, exposure, pix, gout, cfg)
    return L, g, r


def loss_value(m, cams, exposure, targets, pix, cfg=None):
    r = render(m, cams, exposure, pix, cfg)
    rgb, lab, msk = gather_targets(targets, pix)
    L, _ = loss(r.out, rgb, lab, msk, m.num_classes, cfg, grad=False)
    return L, r


def binning(rect, view, key, idx, tile_base, tiles_x, total_tiles):
    """Integer tile lists (CSR) from per-record tile rectangles, each tile's
    records ordered by (binary32 depth key, surfel index)."""
    lib = load()
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    view = np.ascontiguousarray(view, dtype=np.int32)
    key = np.ascontiguousarray(key, dtype=np.float32)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    tb = np.ascontiguousarray(tile_base, dtype=np.int64)
    tx = np.ascontiguousarray(tiles_x, dtype=np.int32)
    offs = np.zeros(total_tiles + 1, np.int64)
    n_rec = rect.shape[0]
    K = lib.orc_bin(C.c_int64(n_rec), _p(rect), _p(view), _p(key), _p(idx), C.c_int(len(tb)), _p(tb), _p(tx),
                    C.c_int64(total_tiles), _p(offs), None)
    lst = np.zeros(max(K, 1), np.int64)
    lib.orc_bin(C.c_int64(n_rec), _p(rect), _p(view), _p(key), _p(idx), C.c_int(len(tb)), _p(tb), _p(tx),
                C.c_int64(total_tiles), _p(offs), _p(lst))
    return offs, lst[:K]


def init_from_poses(xy, poses, exact_plane=True):
    lib = load()
    xy = _f32(xy, (-1, 2))
    poses = _f32(poses, (-1, 12))
    n = xy.shape[0]
    z = np.zeros(n); R = np.zeros((n, 9)); near = np.zeros(n, np.int64)
    rc = lib.orc_init_from_poses(C.c_int64(n), _p(xy), C.c_int64(poses.shape[0]), _p(poses),
                                 C.c_int(1 if exact_plane else 0), _p(z), _p(R), _p(near))
    return rc, z, R.reshape(n, 3, 3), near


def set_threads(n: int):
    load().orc_set_threads(int(n))


def num_threads() -> int:
    return int(load().orc_num_threads())


from .smooth import neighbour_ids, smooth_loss  # noqa: E402,F401
from .adam import adam_step, z_learning_rate  # noqa: E402,F401
from .lidar import elev_loss, nearest_elevation  # noqa: E402,F401
