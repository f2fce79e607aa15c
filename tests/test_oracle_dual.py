"""The oracle's reverse pass against forward-mode derivatives.

A third, independent derivation of the gradient beside the FP64 reverse pass
over stored per-pixel lists and central finite differences: the forward of
RoGs (Eq. 2 with s_z = 0, the EWA projection of Eq. 5 with the 0.3 px^2
low-pass, the front-to-back compositing of Eq. 6 with its alpha clamp,
threshold and stop, the exposure of Eq. 7 and the masked L1 + cross-entropy
loss of Eqs. 8-9) is restated here with dual numbers, each carrying the exact
derivative along K parameter directions at once.  Derivatives through the
discrete decisions (alpha threshold, stop, clamp, Jacobian clamp, sort order)
follow the branch taken at the evaluation point, as a reverse pass does; the
test keeps every pixel the oracle flags as near a threshold out of the loss.

Nothing here shares code with the oracle: only its public render and
loss_and_grads are called.
"""
import numpy as np
import pytest

import oracle
from paper_2405_14342_gb300 import scenes

# the configuration constants are binary32 values (the library's config
# struct holds floats), used here widened to FP64 like every other input
_f = lambda x: float(np.float32(x))
EPS2D = _f(0.3)          # low-pass added to the projected covariance (px^2)
ALPHA_MIN = _f(1.0 / 255.0)
ALPHA_MAX = _f(0.99)
T_MIN = _f(1e-4)
JAC_CLAMP = _f(1.3)
NEAR = _f(0.2)
LAMBDA_C, LAMBDA_S = _f(1.0), _f(0.06)


class Dual:
    """Value v (shape S) with tangents d (shape (K,) + S)."""

    def __init__(self, v, d):
        self.v = np.asarray(v, np.float64)
        d = np.asarray(d, np.float64)
        if d.ndim:   # tangents cover the whole value shape
            d = d.reshape(d.shape[:1] + (1,) * (self.v.ndim - d.ndim + 1) + d.shape[1:])
            d = np.broadcast_to(d, d.shape[:1] + self.v.shape)
        self.d = d

    @staticmethod
    def const(v, K):
        v = np.asarray(v, np.float64)
        return Dual(v, np.zeros((K,) + v.shape))

    def _lift(self, o):
        return o if isinstance(o, Dual) else Dual(np.asarray(o, np.float64), 0.0)

    def tangents(self, nd):
        """Tangents with the value dimensions padded on the left to nd, so that a
        per-surfel quantity (K,) broadcasts against per-pixel ones (K, P)."""
        if self.d.ndim == 0:
            return self.d
        return self.d.reshape(self.d.shape[:1] + (1,) * (nd - self.v.ndim) + self.v.shape)

    def _pair(self, o):
        o = self._lift(o)
        nd = max(self.v.ndim, o.v.ndim)
        return o, self.tangents(nd), o.tangents(nd)

    def __add__(self, o):
        o, da, db = self._pair(o)
        return Dual(self.v + o.v, da + db)

    __radd__ = __add__

    def __neg__(self):
        return Dual(-self.v, -self.d)

    def __sub__(self, o):
        return self + (-self._lift(o))

    def __rsub__(self, o):
        return self._lift(o) + (-self)

    def __mul__(self, o):
        o, da, db = self._pair(o)
        return Dual(self.v * o.v, da * o.v + self.v * db)

    __rmul__ = __mul__

    def __truediv__(self, o):
        o, da, db = self._pair(o)
        return Dual(self.v / o.v, (da * o.v - self.v * db) / (o.v * o.v))

    def __rtruediv__(self, o):
        return self._lift(o) / self


def dexp(x):
    e = np.exp(x.v)
    return Dual(e, x.d * e)


def dlog(x):
    return Dual(np.log(x.v), x.d / x.v)


def dsqrt(x):
    s = np.sqrt(x.v)
    return Dual(s, x.d / (2.0 * s))


def dabs(x):
    return Dual(np.abs(x.v), x.d * np.sign(x.v))


def dwhere(c, a, b):
    nd = max(a.v.ndim, b.v.ndim, np.ndim(c))
    return Dual(np.where(c, a.v, b.v), np.where(c, a.tangents(nd), b.tangents(nd)))


def dclamp(x, lo, hi):
    """Clamp with no derivative where the bound is active."""
    inside = (x.v >= lo) & (x.v <= hi)
    return Dual(np.clip(x.v, lo, hi), np.where(inside, x.d, 0.0))


# ----------------------------------------------------------------- scene

def dual_scene(seed=5, n=80, C=5):
    """Surfels scattered 1.5-3.5 m in front of a pinhole camera and under a
    downward orthographic camera, with generic orientations (unnormalised
    quaternions), anisotropic scales, opacities and features."""
    g = np.random.default_rng(seed)
    xyz = np.stack([g.uniform(1.5, 3.5, n), g.uniform(-1.0, 1.0, n), g.uniform(-0.5, 0.5, n)], -1)
    # four wide surfels beside the pinhole view: the perspective Jacobian is
    # evaluated at the clamped direction for them, and their footprints still
    # reach the image edge
    xyz[-4:] = [[1.6, 1.3, 0.2], [1.7, -1.3, -0.1], [1.6, 0.3, 1.0], [1.8, -0.2, -1.05]]
    quat = g.normal(size=(n, 4)) * g.uniform(0.7, 1.4, size=(n, 1))
    scale = g.uniform(0.05, 0.3, (n, 2))
    scale[-4:] = g.uniform(0.3, 0.4, (4, 2))
    m = scenes.SurfelMap(xyz=xyz.astype(np.float32),
                         scale=scale.astype(np.float32),
                         quat=quat.astype(np.float32),
                         opacity=g.uniform(0.5, 0.98, n).astype(np.float32),
                         rgb=g.uniform(0, 1, (n, 3)).astype(np.float32),
                         sem=g.normal(size=(n, C)).astype(np.float32))
    persp = scenes.make_camera(scenes.PERSP, 64, 48, 60.0, 60.0, scenes.look_rotation(0.0, 0.0),
                               (0.0, 0.0, 0.0), exposure_idx=0)
    ortho = scenes.bev_camera((2.5, 0.0), 64, res_m=0.04, height_m=5.0, ground_z=0.0, exposure_idx=1)
    ortho.height = 48
    ortho.cy = 24.0
    ex = np.array([[0.1, -0.02], [-0.05, 0.03]], np.float32)
    return m, [persp, ortho], ex


def quat_rot(q):
    """Rotation matrix of the normalised quaternion (w, x, y, z), entries as duals."""
    nrm = dsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3])
    w, x, y, z = (qi / nrm for qi in q)
    return [[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]


def project_dual(cam, xyz, scale, quat):
    """Mean, conic and camera depth of one surfel (Eqs. 2, 5)."""
    Rw = np.asarray(cam.R, np.float64)
    tw = np.asarray(cam.t, np.float64)
    p = [xyz[0] * Rw[r, 0] + xyz[1] * Rw[r, 1] + xyz[2] * Rw[r, 2] + tw[r] for r in range(3)]
    if cam.kind == scenes.PERSP:
        u, v = p[0] / p[2], p[1] / p[2]
        mean = (u * cam.fx + cam.cx, v * cam.fy + cam.cy)
        uc = dclamp(u, -JAC_CLAMP * 0.5 * cam.width / cam.fx, JAC_CLAMP * 0.5 * cam.width / cam.fx)
        vc = dclamp(v, -JAC_CLAMP * 0.5 * cam.height / cam.fy, JAC_CLAMP * 0.5 * cam.height / cam.fy)
        J = [[cam.fx / p[2], 0.0, -(uc * cam.fx) / p[2]], [0.0, cam.fy / p[2], -(vc * cam.fy) / p[2]]]
    else:
        mean = (p[0] * cam.fx + cam.cx, p[1] * cam.fy + cam.cy)
        J = [[cam.fx, 0.0, 0.0], [0.0, cam.fy, 0.0]]
    Rq = quat_rot(quat)
    # the surfel's two tangent axes scaled, M = R(q)[:, :2] diag(s_x, s_y), in camera axes
    cols = []
    for k in range(2):
        a_w = [Rq[r][k] * scale[k] for r in range(3)]
        a_c = [a_w[0] * Rw[r, 0] + a_w[1] * Rw[r, 1] + a_w[2] * Rw[r, 2] for r in range(3)]
        cols.append([J[i][0] * a_c[0] + J[i][1] * a_c[1] + J[i][2] * a_c[2] for i in range(2)])
    # Sigma' = T2 T2^T + eps I with T2's columns the projected axes
    s00 = cols[0][0] * cols[0][0] + cols[1][0] * cols[1][0] + EPS2D
    s01 = cols[0][0] * cols[0][1] + cols[1][0] * cols[1][1]
    s11 = cols[0][1] * cols[0][1] + cols[1][1] * cols[1][1] + EPS2D
    det = s00 * s11 - s01 * s01
    conic = (s11 / det, -s01 / det, s00 / det)
    return mean, conic, p[2]


def render_loss_dual(m, cams, ex, tg, pix, seeds):
    """Loss (Eqs. 6-9) over a pixel list with tangents along `seeds`, a list of
    (kind, surfel or view, component) triples."""
    K = len(seeds)

    def param(kind, i, width, values):
        out = []
        for c in range(width):
            d = np.zeros(K)
            for k, s in enumerate(seeds):
                if s == (kind, i, c):
                    d[k] = 1.0
            out.append(Dual(float(values[c]), d))
        return out

    n, C = m.n, m.num_classes
    total = Dual.const(0.0, K)
    n_mask = 0
    per_view = []
    for vi, cam in enumerate(cams):
        sel = pix[:, 0] == vi
        if not sel.any():
            continue
        u = pix[sel, 1].astype(np.float64) + 0.5
        v = pix[sel, 2].astype(np.float64) + 0.5
        # per surfel: projection, features, binary32 depth sort key
        surf = []
        Rw = np.asarray(cam.R, np.float32)
        tw = np.asarray(cam.t, np.float32)
        for i in range(n):
            xyz = param("xyz", i, 3, m.xyz[i].astype(np.float64))
            sc = param("scale", i, 2, m.scale[i].astype(np.float64))
            q = param("quat", i, 4, m.quat[i].astype(np.float64))
            al = param("opacity", i, 1, [float(m.opacity[i])])[0]
            rgb = param("rgb", i, 3, m.rgb[i].astype(np.float64))
            sem = param("sem", i, C, m.sem[i].astype(np.float64))
            mean, conic, depth = project_dual(cam, xyz, sc, q)
            x32 = m.xyz[i].astype(np.float32)
            key = np.float32(np.float32(np.float32(Rw[2, 0] * x32[0]) + np.float32(Rw[2, 1] * x32[1]))
                             + np.float32(Rw[2, 2] * x32[2])) + tw[2]
            if cam.kind == scenes.PERSP and not key > NEAR:
                continue
            surf.append((float(np.float32(key)), i, mean, conic, al, rgb + sem + [depth]))
        surf.sort(key=lambda s_: (s_[0], s_[1]))
        npx = u.shape[0]
        T = Dual.const(np.ones(npx), K)
        done = np.zeros(npx, bool)
        acc = [Dual.const(np.zeros(npx), K) for _ in range(3 + C + 1)]
        for _, i, mean, conic, al, feat in surf:
            dx = Dual(u, 0.0) - mean[0]
            dy = Dual(v, 0.0) - mean[1]
            power = -0.5 * (conic[0] * dx * dx + conic[2] * dy * dy) - conic[1] * dx * dy
            a = al * dexp(power)
            a = dwhere(a.v > ALPHA_MAX, Dual.const(np.full(npx, ALPHA_MAX), K), a)
            keep = (a.v >= ALPHA_MIN) & ~done
            stop = keep & (T.v * (1.0 - a.v) < T_MIN)
            done |= stop
            keep &= ~stop
            zero = Dual.const(np.zeros(npx), K)
            w = dwhere(keep, a * T, zero)
            for ch in range(len(feat)):
                acc[ch] = acc[ch] + w * feat[ch]
            T = dwhere(keep, T * (1.0 - a), T)
        # exposure (Eq. 7): c' = e^a c + b on the colour channels
        ea, eb = param("exposure", cam.exposure_idx, 2, ex[cam.exposure_idx].astype(np.float64))
        rgb_out = [dexp(ea) * acc[ch] + eb for ch in range(3)]
        per_view.append((sel, rgb_out, acc[3:3 + C]))
    for sel, rgb_out, sem_out in per_view:
        rgb_t, lab, msk = oracle.gather_targets(tg, pix[sel])
        mk = msk.astype(bool)
        n_mask += int(mk.sum())
        l1 = Dual.const(np.zeros(mk.shape[0]), len(seeds))
        for ch in range(3):
            l1 = l1 + dabs(rgb_out[ch] - rgb_t[:, ch].astype(np.float64))
        ce = Dual.const(np.zeros(mk.shape[0]), len(seeds))
        if C:
            mx = np.max(np.stack([s_.v for s_ in sem_out]), 0)   # any per-pixel shift works
            se = Dual.const(np.zeros(mk.shape[0]), len(seeds))
            for s_ in sem_out:
                se = se + dexp(s_ - mx)
            lse = dlog(se) + mx
            pick = Dual(np.choose(lab, [s_.v for s_ in sem_out]),
                        np.stack([np.choose(lab, [s_.d[k] for s_ in sem_out]) for k in range(len(seeds))]))
            ce = lse - pick
        term = LAMBDA_C * l1 + LAMBDA_S * ce
        total = total + Dual(np.where(mk, term.v, 0.0).sum(), np.where(mk, term.d, 0.0).sum(-1))
    return Dual(total.v / n_mask, total.d / n_mask)


def test_dual_scene_is_generic():
    """The scene exercises both camera models, overlapping footprints, the stop
    rule and the Jacobian clamp somewhere, so each branch of the derivative is
    visited (checked on the oracle's own forward)."""
    m, cams, ex = dual_scene()
    pix = oracle.full_pixels(cams)
    r = oracle.render(m, cams, ex, pix)
    C = m.num_classes
    for vi in range(len(cams)):
        s = pix[:, 0] == vi
        assert (r.ncomp[s] >= 2).sum() > 200, vi         # overlaps
    assert (r.T < 2e-3).sum() > 20      # T below 0.01: the stop rule can act there
    assert (r.amb != 0).sum() < 10
    assert len(clamped_reaching(m, cams, ex)) >= 2


def clamped_reaching(m, cams, ex):
    """Surfels whose perspective Jacobian is clamped and that reach a pixel of
    the pinhole view."""
    cam = cams[0]
    p = m.xyz.astype(np.float64) @ np.asarray(cam.R, np.float64).T + np.asarray(cam.t, np.float64)
    u, v = p[:, 0] / p[:, 2], p[:, 1] / p[:, 2]
    cl = (np.abs(u) > JAC_CLAMP * 0.5 * cam.width / cam.fx) | (np.abs(v) > JAC_CLAMP * 0.5 * cam.height / cam.fy)
    pix = oracle.full_pixels(cams, views=[0])
    tg = scenes.random_targets(cams, m.num_classes, seed=9)
    _, g, _ = oracle.loss_and_grads(m, cams, ex, tg, pix)
    return [int(i) for i in np.nonzero(cl & (np.abs(g.opacity) > 0))[0]]


def test_reverse_pass_matches_forward_mode():
    m, cams, ex = dual_scene()
    C = m.num_classes
    pix_all = oracle.full_pixels(cams)
    r = oracle.render(m, cams, ex, pix_all)
    pix = pix_all[r.amb == 0]                  # pixels near a threshold stay out of the loss
    tg = scenes.random_targets(cams, C, seed=9)
    L, g, _ = oracle.loss_and_grads(m, cams, ex, tg, pix)
    # parameters of the surfels that reach the most pixels, every kind and component
    reach = np.abs(g.rgb).sum(1)
    top = list(np.argsort(-reach)[:6]) + clamped_reaching(m, cams, ex)[:2]
    seeds = []
    for i in top:
        seeds += [("xyz", int(i), c) for c in range(3)] + [("scale", int(i), c) for c in range(2)]
        seeds += [("quat", int(i), c) for c in range(4)] + [("opacity", int(i), 0)]
        seeds += [("rgb", int(i), c) for c in range(3)] + [("sem", int(i), c) for c in (0, C - 1)]
    seeds += [("exposure", 0, 0), ("exposure", 0, 1), ("exposure", 1, 0), ("exposure", 1, 1)]
    Ld = render_loss_dual(m, cams, ex, tg, pix, seeds)
    assert Ld.v == pytest.approx(L, rel=1e-12)
    rev = np.array([getattr(g, kind).reshape(getattr(g, kind).shape[0], -1)[i, c] for kind, i, c in seeds])
    fwd = Ld.d
    assert np.abs(fwd).max() > 0
    # both are exact derivatives of the same FP64 function: they agree to rounding
    err = np.abs(fwd - rev)
    assert err.max() <= 1e-9 * np.abs(fwd).max(), (err.max(), np.abs(fwd).max())
    for kind in {s[0] for s in seeds}:
        k = np.array([s[0] == kind for s in seeds])
        sc = np.abs(fwd[k]).max()
        assert sc > 0, kind
        assert err[k].max() <= 1e-8 * sc, kind
