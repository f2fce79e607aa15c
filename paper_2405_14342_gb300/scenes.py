"""Seeded synthetic inputs shaped like the paper's road scenes.

This module only *builds inputs*: meshgrid surfel maps (Sec. 3.1, Layout-1),
camera rigs (six surround pinhole cameras, nuScenes-like, Sec. 4.1) and BEV
orthographic cameras (supplementary "Orthogonal Rendering Acceleration",
0.05 m/px).  It holds none of the method's arithmetic: no projection, no
compositing, no loss, no initialisation.  Both the CUDA path and the CPU
oracle consume what it returns, so it depends on numpy only.

Conventions
-----------
* World frame: z up.  Camera frame: x right, y down, z forward.
* A camera is (R_wc, t_wc): p_cam = R_wc @ p_world + t_wc.
* Surfel index = j * nx + i for grid vertex (i, j) at (x0 + s*i, y0 + s*j).
* Quaternions are (w, x, y, z).  The rotation from a surface normal n is the
  minimal rotation taking e_z to n: q = normalise(1 + n_z, -n_y, n_x, 0).
* Seeds: numpy PCG64, parameters seed 0, perturbation seed 1, requests seed 2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

PERSP = 0
ORTHO = 1


@dataclasses.dataclass
class Camera:
    kind: int                 # PERSP or ORTHO
    width: int
    height: int
    fx: float                 # px per unit (ortho: px per metre)
    fy: float
    cx: float
    cy: float
    R: np.ndarray             # (3, 3) float32, world -> camera rotation
    t: np.ndarray             # (3,) float32, world -> camera translation
    exposure_idx: int = 0
    use_box_cull: int = 0

    @property
    def n_pixels(self) -> int:
        return self.width * self.height


@dataclasses.dataclass
class SurfelMap:
    xyz: np.ndarray           # (N, 3) float32
    scale: np.ndarray         # (N, 2) float32, (s_x, s_y) > 0
    quat: np.ndarray          # (N, 4) float32, (w, x, y, z), any norm > 0
    opacity: np.ndarray       # (N,)   float32, alpha in (0, 1]
    rgb: np.ndarray           # (N, 3) float32
    sem: np.ndarray           # (N, C) float32 semantic logits
    grid_shape: tuple = (0, 0)   # (ny, nx) when the map is a full grid

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def num_classes(self) -> int:
        return int(self.sem.shape[1])

    def copy(self) -> "SurfelMap":
        return SurfelMap(self.xyz.copy(), self.scale.copy(), self.quat.copy(), self.opacity.copy(),
                         self.rgb.copy(), self.sem.copy(), tuple(self.grid_shape))


@dataclasses.dataclass
class Targets:
    """Per-view supervision: rgb planes (3,H,W) f32, label (H,W) i32, mask (H,W) u8."""
    rgb: List[np.ndarray]
    label: List[np.ndarray]
    mask: List[np.ndarray]


# ---------------------------------------------------------------- rotations

def quat_from_normal(n: np.ndarray) -> np.ndarray:
    """Minimal rotation e_z -> n as (w,x,y,z), n of shape (...,3), unit."""
    n = np.asarray(n, dtype=np.float64)
    q = np.stack([1.0 + n[..., 2], -n[..., 1], n[..., 0], np.zeros_like(n[..., 0])], axis=-1)
    q /= np.linalg.norm(q, axis=-1, keepdims=True)
    return q


def look_rotation(yaw_deg: float, pitch_down_deg: float) -> np.ndarray:
    """World->camera rotation of a camera with the given yaw (about +z, 0 = +x)
    and downward pitch, camera axes x right, y down, z forward."""
    yaw = math.radians(yaw_deg)
    pit = math.radians(pitch_down_deg)
    fwd = np.array([math.cos(pit) * math.cos(yaw), math.cos(pit) * math.sin(yaw), -math.sin(pit)])
    right = np.array([math.sin(yaw), -math.cos(yaw), 0.0])
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd], axis=0)


def make_camera(kind, width, height, fx, fy, R, centre, exposure_idx=0, use_box_cull=0,
                cx=None, cy=None) -> Camera:
    R64 = np.asarray(R, dtype=np.float64)
    centre = np.asarray(centre, dtype=np.float64)
    t64 = -R64 @ centre
    return Camera(kind=kind, width=int(width), height=int(height), fx=float(fx), fy=float(fy),
                  cx=float(width / 2.0 if cx is None else cx), cy=float(height / 2.0 if cy is None else cy),
                  R=R64.astype(np.float32), t=t64.astype(np.float32),
                  exposure_idx=int(exposure_idx), use_box_cull=int(use_box_cull))


def bev_camera(centre_xy, side_px, res_m=0.05, height_m=100.0, ground_z=0.0, exposure_idx=0) -> Camera:
    """Orthographic camera looking straight down (-z), image x along world +x,
    image y along world -y, res_m metres per pixel."""
    R = np.array([[1.0, 0.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, -1.0]])
    c = np.array([centre_xy[0], centre_xy[1], ground_z + height_m])
    return make_camera(ORTHO, side_px, side_px, 1.0 / res_m, 1.0 / res_m, R, c, exposure_idx=exposure_idx)


# ----------------------------------------------------------- height fields

def height_tiny(x, y):
    z = 0.02 * np.sin(x) * np.cos(y)
    dzdx = 0.02 * np.cos(x) * np.cos(y)
    dzdy = -0.02 * np.sin(x) * np.sin(y)
    return z, dzdx, dzdy


class RandomField:
    """Stationary random height field, RMS `amp`, squared-exponential
    correlation length `corr` (sum of 64 random cosines)."""

    def __init__(self, rng: np.random.Generator, amp=0.1, corr=20.0, n_waves=64):
        self.k = rng.normal(0.0, 1.0 / corr, size=(n_waves, 2))
        self.phi = rng.uniform(0.0, 2.0 * np.pi, size=n_waves)
        self.a = amp * math.sqrt(2.0 / n_waves)

    def __call__(self, x, y, chunk=1 << 20):
        x = np.asarray(x, dtype=np.float64).ravel()
        y = np.asarray(y, dtype=np.float64).ravel()
        z = np.empty_like(x); gx = np.empty_like(x); gy = np.empty_like(x)
        for s in range(0, x.size, chunk):
            xs, ys = x[s:s + chunk, None], y[s:s + chunk, None]
            arg = xs * self.k[None, :, 0] + ys * self.k[None, :, 1] + self.phi[None, :]
            c, sn = np.cos(arg), np.sin(arg)
            z[s:s + chunk] = self.a * c.sum(1)
            gx[s:s + chunk] = -self.a * (sn * self.k[None, :, 0]).sum(1)
            gy[s:s + chunk] = -self.a * (sn * self.k[None, :, 1]).sum(1)
        return z, gx, gy


# ------------------------------------------------------------------ maps

def _assemble(x, y, z, gx, gy, rng, C, opacity=0.9, s=0.06, grid_shape=(0, 0)) -> SurfelMap:
    n = np.stack([-gx, -gy, np.ones_like(gx)], axis=-1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    N = x.size
    return SurfelMap(
        xyz=np.stack([x, y, z], axis=-1).astype(np.float32),
        scale=np.full((N, 2), s, dtype=np.float32),
        quat=quat_from_normal(n).astype(np.float32),
        opacity=np.full((N,), opacity, dtype=np.float32),
        rgb=rng.uniform(0.0, 1.0, size=(N, 3)).astype(np.float32),
        sem=rng.normal(0.0, 1.0, size=(N, C)).astype(np.float32),
        grid_shape=grid_shape,
    )


def grid_xy(nx, ny, x0=0.0, y0=0.0, spacing=0.1):
    i = np.arange(nx, dtype=np.float64)
    j = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x0 + spacing * i, y0 + spacing * j)   # (ny, nx)
    return X.ravel(), Y.ravel()


def tiny_map(C=8, seed=0) -> SurfelMap:
    """64x64 grid at 0.1 m, z = 0.02 sin(x) cos(y)."""
    rng = np.random.default_rng(seed)
    x, y = grid_xy(64, 64)
    z, gx, gy = height_tiny(x, y)
    return _assemble(x, y, z, gx, gy, rng, C, grid_shape=(64, 64))


def tiny_camera() -> Camera:
    R = look_rotation(0.0, 10.0)
    return make_camera(PERSP, 320, 180, 200.0, 200.0, R, (-2.0, 3.15, 1.5), exposure_idx=0, use_box_cull=1)


def strip_map(C=19, seed=0, length=400.0, width=40.0, spacing=0.1):
    """400 x 40 m road strip at 0.1 m spacing (1.6M surfels) on a random field."""
    rng = np.random.default_rng(seed)
    nx, ny = int(round(length / spacing)), int(round(width / spacing))
    field = RandomField(rng)
    x, y = grid_xy(nx, ny, spacing=spacing)
    z, gx, gy = field(x, y)
    return _assemble(x, y, z, gx, gy, rng, C, grid_shape=(ny, nx)), field


def grid_index(m: SurfelMap) -> np.ndarray:
    """Grid -> surfel index map (ny, nx) int32 of a full-grid map (surfel j*nx + i
    sits at grid vertex (j, i)); -1 marks a vertex without a surfel."""
    ny, nx = m.grid_shape
    if ny * nx != m.n:
        raise ValueError("map is not a full grid")
    return np.arange(ny * nx, dtype=np.int32).reshape(ny, nx)


def with_holes(m: SurfelMap, frac: float = 0.2, seed: int = 7):
    """Drop a random fraction of a full-grid map's surfels (off-road vertices),
    keeping the survivors in order; returns the smaller map and its grid index
    map with -1 at the holes."""
    rng = np.random.default_rng(seed)
    gi = grid_index(m)
    keep = rng.uniform(size=m.n) >= frac
    new_id = np.full(m.n, -1, np.int64)
    new_id[keep] = np.arange(int(keep.sum()))
    m2 = SurfelMap(m.xyz[keep].copy(), m.scale[keep].copy(), m.quat[keep].copy(), m.opacity[keep].copy(),
                   m.rgb[keep].copy(), m.sem[keep].copy(), (0, 0))
    return m2, new_id[gi].astype(np.int32)


def lidar_points(height, x_range, y_range, n, noise=0.01, seed=5):
    """Synthetic LiDAR returns on the road: n points uniform in the xy box,
    z = height(x, y) + N(0, noise); float32 [n, 3].  `height` is any callable
    returning the surface height (e.g. a RandomField's first output)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(x_range[0], x_range[1], n)
    y = rng.uniform(y_range[0], y_range[1], n)
    z = np.asarray(height(x, y)) + rng.normal(0.0, noise, n)
    return np.stack([x, y, z], -1).astype(np.float32)


SURROUND_YAWS = (0.0, 55.0, -55.0, 110.0, -110.0, 180.0)


def surround_rig(field, t: int, sizes=None, height=1.5, speed=10.0, hz=12.0, y=20.0, x0=100.0):
    """Six pinhole cameras at timestep t on the straight trajectory y=const.
    `sizes` lists (W, H, hfov_deg) per camera; default 6 x 960x540 with 70 deg
    HFOV and a 110 deg rear camera."""
    if sizes is None:
        sizes = [(960, 540, 70.0)] * 5 + [(960, 540, 110.0)]
    xt = x0 + speed / hz * t
    zg, _, _ = field(np.array([xt]), np.array([y]))
    centre = (xt, y, float(zg[0]) + height)
    cams = []
    for k, (yaw, (W, H, hfov)) in enumerate(zip(SURROUND_YAWS, sizes)):
        f = 0.5 * W / math.tan(math.radians(hfov / 2.0))
        cams.append(make_camera(PERSP, W, H, f, f, look_rotation(yaw, 0.0), centre,
                                exposure_idx=k, use_box_cull=1))
    return cams


BATCH_SIZES = [(1600, 900, 70.0), (1280, 720, 70.0), (1280, 720, 70.0),
               (1280, 720, 70.0), (1280, 720, 70.0), (640, 360, 70.0)]


def grid_road_map(C=19, seed=0, extent=2000.0, lane=3.5, spacing=0.1, roads=(0.0, 1000.0, 2000.0)):
    """2x2 km grid road network: one lane of width `lane` along each road line
    x in roads and y in roads (about 4.19M surfels)."""
    rng = np.random.default_rng(seed)
    field = RandomField(rng)
    n_along = int(round(extent / spacing))
    n_across = int(round(lane / spacing))
    along = np.arange(n_along) * spacing
    across = (np.arange(n_across) - n_across // 2) * spacing
    xs, ys = [], []
    for r in roads:                      # roads parallel to y (x = r)
        X, Y = np.meshgrid(r + across, along)
        xs.append(X.ravel()); ys.append(Y.ravel())
    for r in roads:                      # roads parallel to x (y = r)
        X, Y = np.meshgrid(along, r + across)
        xs.append(X.ravel()); ys.append(Y.ravel())
    x = np.concatenate(xs); y = np.concatenate(ys)
    # a vertex on two roads is kept once (the first occurrence)
    key = np.round(x / spacing).astype(np.int64) * 1_000_003 + np.round(y / spacing).astype(np.int64)
    _, first = np.unique(key, return_index=True)
    first.sort()
    x, y = x[first], y[first]
    z, gx, gy = field(x, y)
    return _assemble(x, y, z, gx, gy, rng, C), field


def intersection_camera(field, at=(1000.0, 1000.0), W=640, H=360, hfov=70.0, pitch=10.0, yaw=0.0):
    zg, _, _ = field(np.array([at[0]]), np.array([at[1]]))
    f = 0.5 * W / math.tan(math.radians(hfov / 2.0))
    return make_camera(PERSP, W, H, f, f, look_rotation(yaw, pitch), (at[0], at[1], float(zg[0]) + 1.5),
                       exposure_idx=0, use_box_cull=1)


def perturb(m: SurfelMap, seed=1, rgb_sigma=0.05, sem_sigma=0.5, z_sigma=0.005) -> SurfelMap:
    """Seed-perturbed copy used to render synthetic supervision targets."""
    rng = np.random.default_rng(seed)
    p = m.copy()
    p.rgb = np.clip(m.rgb + rng.normal(0, rgb_sigma, m.rgb.shape), 0.0, 1.0).astype(np.float32)
    p.sem = (m.sem + rng.normal(0, sem_sigma, m.sem.shape)).astype(np.float32)
    xyz = m.xyz.copy()
    xyz[:, 2] += rng.normal(0, z_sigma, m.n).astype(np.float32)
    p.xyz = xyz.astype(np.float32)
    return p


def exposure_params(n, seed=0, a_sigma=0.05, b_sigma=0.02):
    rng = np.random.default_rng(seed + 100)
    return np.stack([rng.normal(0, a_sigma, n), rng.normal(0, b_sigma, n)], axis=-1).astype(np.float32)


def random_targets(cams: List[Camera], C: int, seed=3, mask_frac=0.8) -> Targets:
    """Unrendered supervision (smooth random images) for tests that only need
    some target of the right shape."""
    rng = np.random.default_rng(seed)
    rgbs, labels, masks = [], [], []
    for c in cams:
        H, W = c.height, c.width
        base = rng.uniform(0, 1, size=(3, 1, 1))
        yy, xx = np.meshgrid(np.linspace(0, 1, H), np.linspace(0, 1, W), indexing="ij")
        rgb = np.clip(base + 0.3 * np.sin(6 * xx + 3 * yy)[None] + rng.normal(0, 0.05, (3, H, W)), 0, 1)
        rgbs.append(rgb.astype(np.float32))
        labels.append(rng.integers(0, C, size=(H, W)).astype(np.int32) if C > 0
                      else np.full((H, W), -1, np.int32))   # no classes: no semantic term
        masks.append((rng.uniform(0, 1, size=(H, W)) < mask_frac).astype(np.uint8))
    return Targets(rgbs, labels, masks)


def camera_arrays(cams: List[Camera]):
    """Flat arrays describing cameras: ints (V,5) = kind, W, H, exposure_idx,
    use_box_cull; floats (V,16) = fx, fy, cx, cy, R (row-major 9), t (3)."""
    ci = np.array([[c.kind, c.width, c.height, c.exposure_idx, c.use_box_cull] for c in cams], dtype=np.int32)
    cf = np.array([[c.fx, c.fy, c.cx, c.cy, *np.asarray(c.R, np.float32).ravel(), *np.asarray(c.t, np.float32)]
                   for c in cams], dtype=np.float32)
    return ci, cf


def poses_on_trajectory(field, n=240, x0=100.0, speed=10.0, hz=12.0, y=20.0, roll_deg=0.0, pitch_deg=0.0):
    """Ground-contact vehicle poses [n,12] = (x,y,z, R row-major) on y=const;
    R columns are the vehicle axes (x forward, y left, z up) in the world."""
    out = np.zeros((n, 12), dtype=np.float32)
    for k in range(n):
        xt = x0 + speed / hz * k
        zg, _, _ = field(np.array([xt]), np.array([y]))
        cr, sr = math.cos(math.radians(roll_deg)), math.sin(math.radians(roll_deg))
        cp, sp = math.cos(math.radians(pitch_deg)), math.sin(math.radians(pitch_deg))
        Rx = np.array([[1, 0, 0], [0, cr, -sr], [0, sr, cr]])
        Ry = np.array([[cp, 0, sp], [0, 1, 0], [-sp, 0, cp]])
        R = Ry @ Rx
        out[k, :3] = (xt, y, float(zg[0]))
        out[k, 3:] = R.ravel()
    return out


def serve_requests(field, n=2000, seed=2, roads=(0.0, 1000.0, 2000.0), extent=2000.0, res_m=0.05):
    """Mixed serving requests over the grid road network: half BEV orthographic
    tiles (side in {256, 512, 1024, 2048} px at res_m, channel set RGB, SEM or
    ELEV) centred on a random road point, half perspective views ({320x180,
    640x360, 1280x720, 1920x1080}, 70 deg HFOV, RGB) at a random road pose.
    Returns a list of (Camera, channels) with channels 1 = RGB, 2 = SEM, 4 = ELEV."""
    rng = np.random.default_rng(seed)
    out = []
    sizes = [(320, 180), (640, 360), (1280, 720), (1920, 1080)]
    for i in range(n):
        along = rng.uniform(50.0, extent - 50.0)
        r = roads[rng.integers(0, len(roads))]
        horizontal = rng.integers(0, 2) == 1           # road along x (y = r) or along y (x = r)
        x, y = (along, r) if horizontal else (r, along)
        zg, _, _ = field(np.array([x]), np.array([y]))
        if i % 2 == 0:
            side = int(rng.choice([256, 512, 1024, 2048]))
            ch = int(rng.choice([1, 2, 4]))
            out.append((bev_camera((x, y), side, res_m=res_m, height_m=100.0, ground_z=float(zg[0])), ch))
        else:
            W, H = sizes[rng.integers(0, 4)]
            yaw = (0.0 if horizontal else 90.0) + (180.0 if rng.integers(0, 2) else 0.0) + rng.normal(0, 3.0)
            f = 0.5 * W / math.tan(math.radians(35.0))
            out.append((make_camera(PERSP, W, H, f, f, look_rotation(yaw, 0.0), (x, y, float(zg[0]) + 1.5),
                                    use_box_cull=1), 1))
    return out
