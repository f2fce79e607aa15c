"""Pins of the oracle's perspective box cull against geometry worked by hand.

Supplementary "Perspective Rendering Acceleration": a perspective camera
renders only the surfels inside a ground box that reaches +-20 m along the
camera's x axis and 0..40 m along its z axis, both axes projected onto the
ground plane, measured from the camera centre.  The reading taken here: the
projected axes are normalised after dropping their height component, and the
box is closed (a surfel exactly on an edge is kept).

The expected decisions below do not use the oracle's formula.  The camera is
built from a yaw, a pitch and a roll, and its ground axes are written down
from those angles:

    z_hat = (cos yaw, sin yaw)                      (pitch only shortens it)
    x_hat = normalise(cos roll (sin yaw, -cos yaw) - sin roll sin pitch (cos yaw, sin yaw))

Surfels are then placed at chosen (lateral, forward) coordinates L, F, i.e.
at o + d with d solving [x_hat; z_hat] d = (L, F); the cull keeps exactly
those with |L| <= 20 and 0 <= F <= 40.  Every placement is at least 5 cm from
an edge, far outside binary32 rounding at these distances.  Mistakes these
pins catch (see test_oracle_mutations.py): the axes swapped, the forward sign
flipped, the 20 m and 40 m sizes swapped, either axis left unnormalised after
the projection, and the camera centre's sign.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

LAT = [-30.0, -20.1, -19.9, -7.0, 0.0, 12.5, 19.9, 20.1, 25.0]
FWD = [-0.1, 0.1, 10.0, 20.5, 30.0, 39.9, 40.1, 40.6, 46.0]
HEIGHT = 1.5


def camera_rotation(yaw_deg, pitch_down_deg, roll_deg):
    """World-to-camera rotation (rows: camera x right, y down, z forward in
    world coordinates, world z up) of a camera with the given heading, downward
    pitch and roll about its viewing axis."""
    y, p, r = (math.radians(a) for a in (yaw_deg, pitch_down_deg, roll_deg))
    fwd = np.array([math.cos(p) * math.cos(y), math.cos(p) * math.sin(y), -math.sin(p)])
    right0 = np.array([math.sin(y), -math.cos(y), 0.0])
    down0 = np.cross(fwd, right0)
    right = math.cos(r) * right0 + math.sin(r) * down0
    down = -math.sin(r) * right0 + math.cos(r) * down0
    return np.stack([right, down, fwd])


def hand_ground_axes(yaw_deg, pitch_down_deg, roll_deg):
    """x_hat, z_hat written down from the angles (see the module docstring)."""
    y, p, r = (math.radians(a) for a in (yaw_deg, pitch_down_deg, roll_deg))
    ex = np.array([math.sin(y), -math.cos(y)])
    ez = np.array([math.cos(y), math.sin(y)])
    xr = math.cos(r) * ex - math.sin(r) * math.sin(p) * ez
    return xr / np.linalg.norm(xr), ez


def box_map(centre_xy, xh, zh, lat=LAT, fwd=FWD):
    """Flat surfels on the ground (z = 0) at every (L, F) of the grid."""
    A = np.stack([xh, zh])                       # [x_hat; z_hat] d = (L, F)
    LF = np.array([(a, b) for a in lat for b in fwd])
    d = np.linalg.solve(A, LF.T).T
    xy = np.asarray(centre_xy)[None, :] + d
    n = len(LF)
    xyz = np.concatenate([xy, np.zeros((n, 1))], 1).astype(np.float32)
    m = scenes.SurfelMap(xyz=xyz, scale=np.full((n, 2), 0.05, np.float32),
                         quat=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                         opacity=np.full(n, 0.9, np.float32), rgb=np.full((n, 3), 0.5, np.float32),
                         sem=np.zeros((n, 1), np.float32))
    keep = (np.abs(LF[:, 0]) <= 20.0) & (LF[:, 1] >= 0.0) & (LF[:, 1] <= 40.0)
    return m, LF, keep


def box_camera(yaw, pitch, roll, centre_xy, box=1, kind=scenes.PERSP, f=150.0):
    R = camera_rotation(yaw, pitch, roll)
    c = scenes.make_camera(kind, 640, 360, f, f, R, (centre_xy[0], centre_xy[1], HEIGHT), use_box_cull=box)
    return c


CASES = [   # yaw, pitch down, roll, camera centre (x, y)
    (35.0, 25.0, 0.0, (53.2, -17.4)),
    (-120.0, 14.0, 10.0, (-8.5, 31.0)),
    (180.0, 30.0, -12.0, (400.25, 20.0)),
    (90.0, 40.0, 0.0, (0.0, 0.0)),
]


@pytest.mark.parametrize("case", CASES)
def test_box_cull_keeps_exactly_the_hand_worked_box(case):
    yaw, pitch, roll, cxy = case
    xh, zh = hand_ground_axes(yaw, pitch, roll)
    m, LF, keep = box_map(cxy, xh, zh)
    cam = box_camera(yaw, pitch, roll, cxy)
    # every placement is in front of the near plane (only the box decides)
    Rc = cam.R.astype(np.float64)
    zc = (m.xyz.astype(np.float64) @ Rc.T + cam.t.astype(np.float64))[:, 2]
    assert (zc > 0.25).all(), zc.min()   # near plane 0.2 m
    vis = oracle.project(m, [cam]).vis[0]
    bad = np.nonzero(vis != keep)[0]
    assert bad.size == 0, [(tuple(LF[i]), bool(keep[i])) for i in bad[:6]]


def test_box_cull_pitched_camera_needs_normalised_forward_axis():
    """Pitched 40 deg down, the forward axis projected to the ground has length
    cos 40 = 0.77: a surfel 40.6 m ahead is outside the box (it would be inside
    at 31 m if the axis were not normalised), 39.9 m is inside."""
    yaw, pitch = 90.0, 40.0
    xh, zh = hand_ground_axes(yaw, pitch, 0.0)
    m, LF, keep = box_map((0.0, 0.0), xh, zh, lat=[0.0], fwd=[39.9, 40.6])
    vis = oracle.project(m, [box_camera(yaw, pitch, 0.0, (0.0, 0.0))]).vis[0]
    np.testing.assert_array_equal(vis, [True, False])


def test_box_cull_rolled_camera_needs_normalised_lateral_axis():
    """Rolled 15 deg and pitched 30 deg, the x axis projected to the ground has
    length sqrt(cos^2 15 + sin^2 15 sin^2 30) = 0.974: 20.1 m to the side is
    outside the box (19.6 m unnormalised)."""
    yaw, pitch, roll = -60.0, 30.0, 15.0
    xh, zh = hand_ground_axes(yaw, pitch, roll)
    m, LF, keep = box_map((5.0, 5.0), xh, zh, lat=[-20.1, 19.9, 20.1], fwd=[10.0])
    vis = oracle.project(m, [box_camera(yaw, pitch, roll, (5.0, 5.0))]).vis[0]
    np.testing.assert_array_equal(vis, [False, True, False])


def test_box_cull_off_and_orthographic_keep_everything_in_front():
    """Without the flag, and for orthographic cameras (which the supplementary
    accelerates by chunking instead), the box culls nothing."""
    yaw, pitch, roll, cxy = CASES[0]
    xh, zh = hand_ground_axes(yaw, pitch, roll)
    m, LF, keep = box_map(cxy, xh, zh)
    vis = oracle.project(m, [box_camera(yaw, pitch, roll, cxy, box=0)]).vis[0]
    assert vis.all()
    bev = scenes.bev_camera(cxy, 64, res_m=0.05)
    bev.use_box_cull = 1
    assert oracle.project(m, [bev]).vis[0].all()
