"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms for special geometries (Eqs. 2, 5 with s_z = 0), two-surfel
compositing (Eq. 6), the blend-weight invariant, in-plane rotation
invariance, the exposure model (Eq. 7), the loss definitions (Eqs. 8-9),
the plane-constrained initialisation (Eq. 4, Eqs. S1-S2), brute-force tile
lists and central finite differences for the gradient.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

ALPHA_MIN = np.float32(1.0 / 255.0)
EPS = 0.3


def one_map(xyz, quat, scale, opacity, rgb, sem):
    xyz = np.asarray(xyz, np.float32).reshape(-1, 3)
    n = xyz.shape[0]
    return scenes.SurfelMap(xyz=xyz, scale=np.asarray(scale, np.float32).reshape(n, 2),
                            quat=np.asarray(quat, np.float32).reshape(n, 4),
                            opacity=np.asarray(opacity, np.float32).reshape(n),
                            rgb=np.asarray(rgb, np.float32).reshape(n, 3),
                            sem=np.asarray(sem, np.float32).reshape(n, -1))


def quat_of_matrix(R):
    """(w,x,y,z) of a rotation matrix (test-side helper, trace method)."""
    R = np.asarray(R, np.float64)
    w = math.sqrt(max(0.0, 1.0 + R[0, 0] + R[1, 1] + R[2, 2])) / 2.0
    x = math.copysign(math.sqrt(max(0.0, 1.0 + R[0, 0] - R[1, 1] - R[2, 2])) / 2.0, R[2, 1] - R[1, 2])
    y = math.copysign(math.sqrt(max(0.0, 1.0 - R[0, 0] + R[1, 1] - R[2, 2])) / 2.0, R[0, 2] - R[2, 0])
    z = math.copysign(math.sqrt(max(0.0, 1.0 - R[0, 0] - R[1, 1] + R[2, 2])) / 2.0, R[1, 0] - R[0, 1])
    return np.array([w, x, y, z])


def cam_from_rotation(R, centre, W=200, H=150, f=180.0, cx=97.3, cy=71.6, kind=scenes.PERSP):
    R32 = np.asarray(R, np.float32)
    t = (-R32.astype(np.float64) @ np.asarray(centre, np.float64)).astype(np.float32)
    return scenes.Camera(kind=kind, width=W, height=H, fx=f, fy=f, cx=cx, cy=cy, R=R32, t=t,
                         exposure_idx=0, use_box_cull=0)


def expected_single(mu, cov, alpha, colour, W, H):
    """c * min(0.99, alpha * g) where alpha*g >= 1/255 (one surfel, Eq. 6)."""
    vv, uu = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    dx, dy = uu - mu[0], vv - mu[1]
    a_, b_, c_ = cov
    det = a_ * c_ - b_ * b_
    power = -0.5 * (c_ * dx * dx - 2 * b_ * dx * dy + a_ * dy * dy) / det
    a = np.minimum(0.99, alpha * np.exp(power))
    a = np.where(alpha * np.exp(power) >= float(ALPHA_MIN), a, 0.0)
    return a[..., None] * np.asarray(colour)[None, None, :], a


def frame(r, cam, C):
    return r.out.reshape(cam.height, cam.width, 3 + C + 1)


# ------------------------------------------------------------------ Eq. 2, 5

def test_fronto_parallel_surfel_closed_form():
    """A surfel whose axes are the camera's axes has Sigma_cam = diag(sx^2, sy^2, 0),
    so Sigma_2D = diag((f sx/z)^2, (f sy/z)^2) + eps I and mu = (f x/z + cx, f y/z + cy)."""
    R = scenes.look_rotation(33.0, 21.0)               # generic camera rotation
    centre = np.array([3.0, -2.0, 4.0])
    cam = cam_from_rotation(R, centre)
    Rc = cam.R.astype(np.float64)
    # surfel axes = camera axes in the world: R_q = R_wc^T
    q = quat_of_matrix(Rc.T)
    for pc in ([0.0, 0.0, 6.0], [0.7, -0.4, 5.0]):
        pw = (Rc.T @ (np.asarray(pc) - cam.t.astype(np.float64)))
        m = one_map(pw, q, [0.05, 0.11], 0.8, [0.2, 0.5, 0.9], [1.0, -2.0])
        r = oracle.render(m, [cam], np.zeros((1, 2)), oracle.full_pixels([cam]))
        # exact camera-space point of the float32 input
        p = Rc @ m.xyz[0].astype(np.float64) + cam.t.astype(np.float64)
        z = p[2]
        f = cam.fx
        mu = (f * p[0] / z + cam.cx, f * p[1] / z + cam.cy)
        sx, sy = 0.05, 0.11
        # R_q from a float32 quaternion is orthonormal only to ~1e-7
        cov = ((f * np.float32(sx) / z) ** 2 + EPS, 0.0, (f * np.float32(sy) / z) ** 2 + EPS)
        exp_rgb, a = expected_single(mu, cov, 0.8, m.rgb[0].astype(np.float64), cam.width, cam.height)
        got = frame(r, cam, 2)
        assert np.abs(got[..., :3] - exp_rgb).max() < 2e-6
        exp_sem = a[..., None] * m.sem[0].astype(np.float64)[None, None, :]
        assert np.abs(got[..., 3:5] - exp_sem).max() < 4e-6
        assert np.abs(got[..., 5] - a * z).max() < 1e-5


def test_tilted_surfel_uses_jacobian_third_column():
    """A surfel tilted about the camera x axis by phi, seen off-axis: Sigma_2D =
    T2 T2^T + eps I with T2 columns J(sx,0,0) and J sy(0,cos phi,sin phi)."""
    R = scenes.look_rotation(-20.0, 12.0)
    cam = cam_from_rotation(R, [1.0, 2.0, 1.5])
    Rc = cam.R.astype(np.float64)
    phi = 0.9
    axes_cam = np.array([[1, 0, 0], [0, math.cos(phi), -math.sin(phi)], [0, math.sin(phi), math.cos(phi)]])
    Rq = Rc.T @ axes_cam                                   # surfel axes in the world
    pc = np.array([0.9, 0.6, 4.0])
    pw = Rc.T @ (pc - cam.t.astype(np.float64))
    sx, sy = 0.07, 0.05
    m = one_map(pw, quat_of_matrix(Rq), [sx, sy], 0.7, [1, 1, 1], [0.0])
    r = oracle.render(m, [cam], np.zeros((1, 2)), oracle.full_pixels([cam]))
    p = Rc @ m.xyz[0].astype(np.float64) + cam.t.astype(np.float64)
    x, y, z = p
    f = cam.fx
    col0 = np.array([f * sx / z, 0.0])
    col1 = sy * np.array([-f * x * math.sin(phi) / z ** 2,
                          f * math.cos(phi) / z - f * y * math.sin(phi) / z ** 2])
    S = np.outer(col0, col0) + np.outer(col1, col1) + EPS * np.eye(2)
    mu = (f * x / z + cam.cx, f * y / z + cam.cy)
    exp_rgb, _ = expected_single(mu, (S[0, 0], S[0, 1], S[1, 1]), 0.7, [1.0, 1.0, 1.0], cam.width, cam.height)
    got = frame(r, cam, 1)
    assert np.abs(got[..., 0] - exp_rgb[..., 0]).max() < 5e-6


def test_ortho_flat_road_closed_form():
    """Orthographic camera looking down (J = pixel scale): a flat surfel rotated
    by theta about z has Sigma_2D = f^2 Rot(-theta) diag(sx^2, sy^2) Rot(-theta)^T + eps I
    (image y points to world -y) and mu = (f (x-cx_w) + cx, -f (y-cy_w) + cy)."""
    cam = scenes.bev_camera((10.0, 20.0), 64, res_m=0.05)
    theta = 0.6
    q = np.array([math.cos(theta / 2), 0, 0, math.sin(theta / 2)])
    sx, sy = 0.12, 0.05
    pw = [10.3, 19.6, 0.02]
    m = one_map(pw, q, [sx, sy], 0.9, [0.3, 0.6, 0.1], [0.5])
    r = oracle.render(m, [cam], np.zeros((1, 2)), oracle.full_pixels([cam]))
    f = 1.0 / 0.05
    c, s = math.cos(theta), math.sin(theta)
    Rimg = np.array([[c, -s], [-s, -c]])                  # world xy axes -> image axes, y flipped
    S = f * f * Rimg @ np.diag([np.float32(sx) ** 2, np.float32(sy) ** 2]) @ Rimg.T + EPS * np.eye(2)
    xyz = m.xyz[0].astype(np.float64)
    mu = (f * (xyz[0] - 10.0) + 32.0, -f * (xyz[1] - 20.0) + 32.0)
    exp_rgb, a = expected_single(mu, (S[0, 0], S[0, 1], S[1, 1]), 0.9, m.rgb[0].astype(np.float64), 64, 64)
    got = frame(r, cam, 1)
    assert np.abs(got[..., :3] - exp_rgb).max() < 1e-5
    # depth = camera z = 100 - z_w for this camera
    assert np.abs(got[..., 4] - a * (100.0 - xyz[2])).max() < 1e-4


def test_projection_table_matches_closed_form():
    R = scenes.look_rotation(0.0, 0.0)
    cam = cam_from_rotation(R, [0.0, 0.0, 0.0])
    Rc = cam.R.astype(np.float64)
    q = quat_of_matrix(Rc.T)
    m = one_map([5.0, 0.0, 0.0], q, [0.1, 0.1], 0.9, [1, 1, 1], [0.0])
    pr = oracle.project(m, [cam])
    assert pr.vis[0, 0]
    z = 5.0
    exp = (cam.fx * 0.1 / z) ** 2 + EPS
    np.testing.assert_allclose(pr.cov[0, 0], [exp, 0.0, exp], atol=1e-5)
    np.testing.assert_allclose(pr.con[0, 0], [1 / exp, 0.0, 1 / exp], rtol=1e-5)
    np.testing.assert_allclose(pr.mu[0, 0], [cam.cx, cam.cy], atol=1e-6)
    assert abs(pr.depth[0, 0] - 5.0) < 1e-6


# --------------------------------------------------------------- Eq. 6

def _two(depths, idx_order=(0, 1), alphas=(0.7, 0.5)):
    R = scenes.look_rotation(0.0, 0.0)
    cam = cam_from_rotation(R, [0.0, 0.0, 0.0], W=40, H=30, cx=20.0, cy=15.0)
    Rc = cam.R.astype(np.float64)
    q = quat_of_matrix(Rc.T)
    pts = [Rc.T @ np.array([0.0, 0.0, d]) for d in depths]
    cols = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]]
    order = list(idx_order)
    m = one_map([pts[k] for k in order], [q, q], [[0.05, 0.05]] * 2, [alphas[k] for k in order],
                [cols[k] for k in order], [[0.0]] * 2)
    return cam, m


@pytest.mark.parametrize("idx_order", [(0, 1), (1, 0)])
def test_two_surfel_compositing_closed_form(idx_order):
    """C = c1 a1 + c2 a2 (1-a1), T = (1-a1)(1-a2), whatever the index order."""
    cam, m = _two([3.0, 4.0], idx_order)
    pix = oracle.full_pixels([cam])
    r = oracle.render(m, [cam], np.zeros((1, 2)), pix)
    f = cam.fx
    a = []
    for d, al in ((3.0, 0.7), (4.0, 0.5)):
        s2 = (f * np.float32(0.05) / d) ** 2 + EPS
        _, ak = expected_single((cam.cx, cam.cy), (s2, 0.0, s2), al, [1, 1, 1], cam.width, cam.height)
        a.append(ak)
    exp_r = a[0]
    exp_g = a[1] * (1 - a[0])
    got = frame(r, cam, 1)
    assert np.abs(got[..., 0] - exp_r).max() < 1e-5
    assert np.abs(got[..., 1] - exp_g).max() < 1e-5
    assert np.abs(r.T.reshape(cam.height, cam.width) - (1 - a[0]) * (1 - a[1])).max() < 1e-5


def test_equal_depth_breaks_ties_by_index():
    cam, m = _two([3.0, 3.0], (1, 0))       # index 0 carries colour green, alpha 0.5
    r = oracle.render(m, [cam], np.zeros((1, 2)), oracle.full_pixels([cam]))
    got = frame(r, cam, 1)
    f = cam.fx
    s2 = (f * np.float32(0.05) / 3.0) ** 2 + EPS
    _, a_g = expected_single((cam.cx, cam.cy), (s2, 0, s2), 0.5, [1, 1, 1], cam.width, cam.height)
    _, a_r = expected_single((cam.cx, cam.cy), (s2, 0, s2), 0.7, [1, 1, 1], cam.width, cam.height)
    # lower index (green, 0.5) first
    assert np.abs(got[..., 1] - a_g).max() < 1e-5
    assert np.abs(got[..., 0] - a_r * (1 - a_g)).max() < 1e-5


def test_early_stop_excludes_the_surfel_that_crosses_t_min():
    """Four surfels with a ~ 0.95 at one pixel: T goes 1 -> 5e-2 -> 2.5e-3 ->
    1.3e-4; the fourth would take T to ~6e-6 < t_min, so it is not composited."""
    R = scenes.look_rotation(0.0, 0.0)
    cam = cam_from_rotation(R, [0.0, 0.0, 0.0], W=8, H=8, cx=4.0, cy=4.0)
    Rc = cam.R.astype(np.float64)
    q = quat_of_matrix(Rc.T)
    depths = (2.0, 2.5, 3.0, 3.5)
    pts = [Rc.T @ np.array([0.0, 0.0, d]) for d in depths]
    cols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float64)
    m = one_map(pts, [q] * 4, [[0.5, 0.5]] * 4, [0.95] * 4, cols, [[0.0]] * 4)
    r = oracle.render(m, [cam], np.zeros((1, 2)), np.array([[0, 4, 4]], np.int32))
    a = []
    for d in depths:
        s2 = (cam.fx * 0.5 / d) ** 2 + EPS
        a.append(float(np.float32(0.95)) * math.exp(-0.5 * (0.25 + 0.25) / s2))
    T = [1.0]
    for ak in a:
        T.append(T[-1] * (1 - ak))
    assert T[3] > 1e-4 > T[4]
    assert r.ncomp[0] == 3 and r.amb[0] == 0
    exp = sum(a[k] * T[k] * cols[k] for k in range(3))
    np.testing.assert_allclose(r.out[0, :3], exp, rtol=1e-9)
    assert abs(r.T[0] - T[3]) < 1e-12


def test_blend_weights_plus_transmittance_is_one():
    m = scenes.tiny_map()
    cam = scenes.tiny_camera()
    r = oracle.render(m, [cam], np.zeros((1, 2)), oracle.full_pixels([cam]))
    assert np.abs(r.sumw + r.T - 1.0).max() < 1e-12
    assert (r.T >= 1e-4).all()
    assert r.T.min() < 0.01           # the map does cover part of the frame


def test_inplane_rotation_invariance_for_isotropic_surfels():
    m = scenes.tiny_map()
    cam = scenes.tiny_camera()
    pix = oracle.full_pixels([cam])
    r0 = oracle.render(m, [cam], np.zeros((1, 2)), pix)
    rng = np.random.default_rng(5)
    th = rng.uniform(0, 2 * np.pi, m.n)
    qz = np.stack([np.cos(th / 2), 0 * th, 0 * th, np.sin(th / 2)], -1)
    q = m.quat.astype(np.float64)
    w1, x1, y1, z1 = q.T
    w2, x2, y2, z2 = qz.T
    prod = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], -1)
    m2 = m.copy()
    m2.quat = prod.astype(np.float32)
    r1 = oracle.render(m2, [cam], np.zeros((1, 2)), pix)
    ok = (r0.amb == 0) & (r1.amb == 0)
    assert np.abs(r0.out[ok] - r1.out[ok]).max() < 1e-5


# --------------------------------------------------------------- Eq. 7

def test_exposure_is_affine_in_the_composite():
    m = scenes.tiny_map()
    cam = scenes.tiny_camera()
    pix = oracle.full_pixels([cam])
    r0 = oracle.render(m, [cam], np.zeros((1, 2)), pix)
    a, b = 0.3, -0.07
    r1 = oracle.render(m, [cam], np.array([[a, b]], np.float32), pix)
    np.testing.assert_allclose(r1.out[:, :3], math.exp(np.float32(a)) * r0.out[:, :3] + np.float32(b),
                               atol=1e-12)
    np.testing.assert_array_equal(r1.out[:, 3:], r0.out[:, 3:])
    # d/db of sum(out_rgb) = 3 * n_pix, d/da = sum(e^a * raw)
    gout = np.zeros_like(r1.out)
    gout[:, :3] = 1.0
    g = oracle.backward(m, [cam], np.array([[a, b]], np.float32), pix, gout)
    assert abs(g.exposure[0, 1] - 3 * len(pix)) < 1e-9
    assert abs(g.exposure[0, 0] - math.exp(np.float32(a)) * r0.out[:, :3].sum()) < 1e-6


# ------------------------------------------------------------- Eqs. 8, 9

def test_loss_closed_form():
    C_ = 3
    out = np.array([[0.5, 0.2, 0.75, 1.0, 2.0, 0.5, 7.0],
                    [0.1, 0.1, 0.1, 0.0, 0.0, 0.0, 1.0],
                    [0.4, 0.4, 0.4, 3.0, -1.0, 0.0, 2.0]])
    tgt = np.array([[0.4, 0.4, 0.75], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]], np.float32)
    label = np.array([1, 0, 2], np.int32)
    mask = np.array([1, 0, 1], np.uint8)
    cfg = oracle.cfg_array(lambda_c=1.0, lambda_s=0.06)
    L, g = oracle.loss(out, tgt, label, mask, C_, cfg)
    t = tgt.astype(np.float64)
    l1 = (abs(0.5 - t[0, 0]) + abs(0.2 - t[0, 1]) + 0.0 + 0.4 * 3) / 2
    lse0 = math.log(math.e ** 1 + math.e ** 2 + math.e ** 0.5)
    lse2 = math.log(math.e ** 3 + math.e ** -1 + 1)
    ce = ((lse0 - 2.0) + (lse2 - 0.0)) / 2
    assert abs(L - (l1 + np.float32(0.06) * ce)) < 1e-7
    assert g[1].max() == 0 and g[1].min() == 0          # unmasked pixel
    np.testing.assert_allclose(g[0, :3], [0.5, -0.5, 0.0], atol=1e-8)   # sign(0) = 0
    sm = np.exp(out[2, 3:6] - lse2)
    np.testing.assert_allclose(g[2, 3:6], np.float32(0.06) / 2 * (sm - np.array([0, 0, 1])), atol=1e-8)
    assert (g[:, 6] == 0).all()                         # depth is not supervised
    # finite differences of the loss w.r.t. out
    e = 1e-6
    for (p, ch) in [(0, 3), (2, 4), (0, 0), (2, 1)]:
        o1 = out.copy(); o1[p, ch] += e
        o2 = out.copy(); o2[p, ch] -= e
        fd = (oracle.loss(o1, tgt, label, mask, C_, cfg, grad=False)[0] -
              oracle.loss(o2, tgt, label, mask, C_, cfg, grad=False)[0]) / (2 * e)
        assert abs(fd - g[p, ch]) < 1e-6


def test_loss_with_empty_mask_is_zero():
    out = np.ones((4, 6))
    L, g = oracle.loss(out, np.zeros((4, 3)), np.zeros(4, np.int32), np.zeros(4, np.uint8), 2)
    assert L == 0.0 and not g.any()


# -------------------------------------------------------- Eq. 4, S1, S2

def test_init_on_tilted_plane_is_exact():
    """Poses on z = z0 + a x + b y with n3 the plane normal: every init z lies
    on that plane (Eq. S1), and R = R_v."""
    a, b, z0 = 0.03, -0.02, 1.2
    n3 = np.array([-a, -b, 1.0]); n3 /= np.linalg.norm(n3)
    e1 = np.array([1.0, 0.0, a]); e1 -= n3 * (e1 @ n3); e1 /= np.linalg.norm(e1)
    e2 = np.cross(n3, e1)
    Rv = np.stack([e1, e2, n3], axis=1)                   # columns n1 n2 n3
    P = 7
    poses = np.zeros((P, 12), np.float32)
    for k in range(P):
        x, y = 5.0 * k, 1.0 + 0.5 * k
        poses[k, :3] = (x, y, z0 + a * x + b * y)
        poses[k, 3:] = Rv.ravel()
    rng = np.random.default_rng(0)
    xy = rng.uniform(-5, 35, size=(500, 2)).astype(np.float32)
    rc, z, R, near = oracle.init_from_poses(xy, poses, exact_plane=True)
    assert rc == 0
    # plane through each used pose with the float32 normal
    for i in range(0, 500, 37):
        pv = poses[near[i]].astype(np.float64)
        n = pv[3:].reshape(3, 3)[:, 2]
        d = n @ np.array([xy[i, 0] - pv[0], xy[i, 1] - pv[1], z[i] - pv[2]])
        assert abs(d) < 1e-12
        np.testing.assert_array_equal(R[i], poses[near[i], 3:].reshape(3, 3).astype(np.float64))
    # globally: all points near the analytic plane (float32 pose rounding only)
    assert np.abs(z - (z0 + a * xy[:, 0].astype(np.float64) + b * xy[:, 1])).max() < 1e-5


def test_init_yaw_only_and_small_roll_reading():
    P = 4
    poses = np.zeros((P, 12), np.float32)
    for k in range(P):
        yaw = 0.3 * k
        Rz = np.array([[math.cos(yaw), -math.sin(yaw), 0], [math.sin(yaw), math.cos(yaw), 0], [0, 0, 1]])
        poses[k, :3] = (10.0 * k, 0.0, 0.5 * k)
        poses[k, 3:] = Rz.ravel()
    xy = np.array([[3.0, 1.0], [7.0, -2.0], [5.0, 0.0], [25.0, 3.0], [100.0, 0.0]], np.float32)
    rc, z, R, near = oracle.init_from_poses(xy, poses, exact_plane=True)
    np.testing.assert_array_equal(near, [0, 1, 0, 2, 3])    # x=5 is a tie -> lowest index
    np.testing.assert_allclose(z, 0.5 * near, atol=1e-7)
    # small-roll reading: z = z_v whatever the tilt
    poses2 = poses.copy()
    poses2[:, 3:] = np.array([[1, 0, 0], [0, 0.9, -0.43589], [0, 0.43589, 0.9]], np.float32).ravel()
    _, z2, _, _ = oracle.init_from_poses(xy, poses2, exact_plane=False)
    np.testing.assert_allclose(z2, 0.5 * near, atol=1e-7)
    _, z3, _, _ = oracle.init_from_poses(xy, poses2, exact_plane=True)
    assert np.abs(z3 - z2).max() > 0.1                        # the exact plane does tilt


def test_init_rejects_vertical_normal():
    poses = np.zeros((1, 12), np.float32)
    poses[0, 3:] = np.array([[1, 0, 0], [0, 0, -1], [0, 1, 0]], np.float32).ravel()   # n33 = 0
    rc, *_ = oracle.init_from_poses(np.zeros((2, 2), np.float32), poses, exact_plane=True)
    assert rc == -1


# ------------------------------------------------------------- binning

def test_binning_hand_example():
    # two views: view 0 2x2 tiles, view 1 3x1 tiles
    tile_base = np.array([0, 4]); tiles_x = np.array([2, 3]); total = 7
    rect = np.array([[0, 0, 1, 0], [1, 0, 1, 1], [0, 0, 0, 0], [0, 0, 2, 0], [1, 0, 1, 0]])
    view = np.array([0, 0, 0, 1, 1])
    key = np.array([2.0, 1.0, 2.0, 5.0, 5.0], np.float32)
    idx = np.array([9, 4, 3, 8, 2])
    offs, lst = oracle.binning(rect, view, key, idx, tile_base, tiles_x, total)
    lists = [list(lst[offs[t]:offs[t + 1]]) for t in range(total)]
    assert lists == [[2, 0], [1, 0], [], [1], [3], [4, 3], [3]]


def conservative_rects(pr, cam, tw=16, th=16, alpha=0.9):
    kappa = 2 * np.log(alpha / float(ALPHA_MIN))
    rx = np.sqrt(kappa * pr.cov[0, :, 0]) * 1.001 + 1e-3
    ry = np.sqrt(kappa * pr.cov[0, :, 2]) * 1.001 + 1e-3
    mu = pr.mu[0]
    x0 = np.floor((mu[:, 0] - rx - 0.5) / tw); x1 = np.floor((mu[:, 0] + rx - 0.5) / tw)
    y0 = np.floor((mu[:, 1] - ry - 0.5) / th); y1 = np.floor((mu[:, 1] + ry - 0.5) / th)
    tx, ty = -(-cam.width // tw), -(-cam.height // th)
    ok = pr.vis[0] & (x1 >= 0) & (y1 >= 0) & (x0 <= tx - 1) & (y0 <= ty - 1)
    r = np.stack([np.clip(x0, 0, tx - 1), np.clip(y0, 0, ty - 1), np.clip(x1, 0, tx - 1), np.clip(y1, 0, ty - 1)], -1)
    return r.astype(np.int32), ok, tx, ty


def test_brute_force_contributors_lie_in_their_tile_lists():
    """Every surfel the brute-force renderer composites at a pixel appears in
    the conservative tile list of that pixel's tile (the tiling changes nothing)."""
    m = scenes.tiny_map()
    cam = scenes.tiny_camera()
    pr = oracle.project(m, [cam])
    rect, ok, tx, ty = conservative_rects(pr, cam)
    ids = np.nonzero(ok)[0]
    offs, lst = oracle.binning(rect[ids], np.zeros(len(ids)), pr.key[0, ids], ids, [0], [tx], tx * ty)
    members = [set(ids[lst[offs[t]:offs[t + 1]]]) for t in range(tx * ty)]
    pix = oracle.full_pixels([cam])
    r = oracle.render(m, [cam], np.zeros((1, 2)), pix)
    sel = np.nonzero(r.last >= 0)[0]
    for p in sel[:: max(1, len(sel) // 4000)]:
        u, v = pix[p, 1], pix[p, 2]
        assert r.last[p] in members[(v // 16) * tx + u // 16]
    # and each tile's list is sorted by (key, index)
    for t in range(tx * ty):
        s = ids[lst[offs[t]:offs[t + 1]]]
        k = pr.key[0, s]
        assert all((k[i], s[i]) < (k[i + 1], s[i + 1]) for i in range(len(s) - 1))


# ---------------------------------------------------- gradient vs FD

def _fd_setup():
    """Tiny scene made generic: anisotropic scales, random in-plane rotations and
    opacities (so that no quaternion component or scale symmetry is zero)."""
    m = scenes.tiny_map()
    g = np.random.default_rng(3)
    m.scale = (0.06 * g.uniform(0.7, 1.3, size=(m.n, 2))).astype(np.float32)
    th = g.uniform(0, 2 * np.pi, m.n)
    q = m.quat.astype(np.float64)
    w1, x1, y1, z1 = q.T
    w2, z2 = np.cos(th / 2), np.sin(th / 2)
    m.quat = np.stack([w1 * w2 - z1 * z2, x1 * w2 + y1 * z2, y1 * w2 - x1 * z2, w1 * z2 + z1 * w2], -1)
    m.quat = (m.quat * g.uniform(0.8, 1.2, size=(m.n, 1))).astype(np.float32)   # unnormalised on purpose
    m.opacity = g.uniform(0.5, 0.98, size=m.n).astype(np.float32)
    cam = scenes.tiny_camera()
    ex = np.array([[0.1, -0.02]], np.float32)
    pix = oracle.crop_pixels(0, 150, 110, 24, 16)
    rng = np.random.default_rng(7)
    H, W = cam.height, cam.width
    tg = scenes.Targets([rng.uniform(0, 1, (3, H, W)).astype(np.float32)],
                        [rng.integers(0, m.num_classes, (H, W)).astype(np.int32)],
                        [(rng.uniform(0, 1, (H, W)) < 0.8).astype(np.uint8)])
    return m, cam, ex, pix, tg


def _perturbed(m, name, i, k, d):
    m2 = m.copy()
    arr = getattr(m2, name).astype(np.float64)
    flat = arr.reshape(arr.shape[0], -1)
    flat[i, k] += d
    setattr(m2, name, flat.reshape(arr.shape))
    return m2


def test_gradient_matches_central_differences():
    """FP64 reverse pass vs central differences of the FP64 forward.  The
    parameters are held in float64 during the FD sweep so that the +-eps
    perturbation is exact."""
    m, cam, ex, pix, tg = _fd_setup()
    L, g, r = oracle.loss_and_grads(m, [cam], ex, tg, pix)
    # surfels that matter for the crop
    hit = np.unique(np.abs(g.rgb).sum(1).nonzero()[0])
    assert len(hit) > 20
    rng = np.random.default_rng(11)
    chosen = rng.choice(hit, size=12, replace=False)
    eps = 1e-4
    base_sig = r.sig.copy()
    rows = []
    for i in chosen:
        for name, k in [("xyz", 0), ("xyz", 1), ("xyz", 2), ("scale", 0), ("scale", 1), ("quat", 0),
                        ("quat", 1), ("quat", 2), ("quat", 3), ("opacity", 0), ("rgb", 1), ("sem", 3)]:
            vals = []
            flip = False
            for d in (+eps, -eps):
                mp = _perturbed(m, name, i, k, d)
                Lp, rp = oracle.loss_value(mp, [cam], ex, tg, pix)
                # a perturbation that reorders or changes a composited list crosses a
                # discontinuity of the forward: such samples are excluded and counted
                flip |= not np.array_equal(rp.sig, base_sig)
                vals.append(Lp)
            if flip:
                continue
            fd = (vals[0] - vals[1]) / (2 * eps)
            an = getattr(g, name).reshape(m.n, -1)[i, k]
            rows.append((name, fd, an))
    assert len(rows) > 100
    fd = np.array([r_[1] for r_ in rows]); an = np.array([r_[2] for r_ in rows])
    scale = np.abs(fd).max()
    assert np.abs(fd - an).max() / scale < 1e-4
    # per parameter kind
    for name in {r_[0] for r_ in rows}:
        s = np.array([r_[0] == name for r_ in rows])
        sc = max(np.abs(fd[s]).max(), 1e-12)
        assert np.abs(fd[s] - an[s]).max() / sc < 1e-3, name
    # exposure
    for k in (0, 1):
        vals = []
        for d in (+eps, -eps):
            e2 = ex.astype(np.float64).copy(); e2[0, k] += d
            vals.append(oracle.loss_value(m, [cam], e2, tg, pix)[0])
        fd_e = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd_e - g.exposure[0, k]) < 1e-4 * max(1.0, abs(fd_e))
