"""PyTorch front end of librogs: device memory, streams and autograd only.

Every step of the method (projection, binning and sorting, compositing,
loss, backward, initialisation) runs in librogs' CUDA kernels through the
C-ABI binding in ``rogs``; this module allocates tensors, passes pointers and
wraps the forward/backward pair in a ``torch.autograd.Function``.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import rogs as R


@dataclasses.dataclass
class SurfelTensors:
    """Device copy of a surfel map (Sec. 3.1, Eq. 3): xyz [N,3], scale [N,2],
    quat [N,4], opacity [N], rgb [N,3], sem [N,C] (FP32, contiguous), and
    optionally the grid index map [H,W] int32 (surfel per grid vertex, -1 off
    the road) used by the smoothness loss."""
    xyz: torch.Tensor
    scale: torch.Tensor
    quat: torch.Tensor
    opacity: torch.Tensor
    rgb: torch.Tensor
    sem: torch.Tensor
    grid_index: torch.Tensor = None

    @staticmethod
    def from_map(m, device="cuda", grid_index=None) -> "SurfelTensors":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=device).contiguous()
        gi = None
        if grid_index is not None:
            gi = torch.as_tensor(np.ascontiguousarray(grid_index, dtype=np.int32), device=device).contiguous()
        return SurfelTensors(f(m.xyz), f(m.scale), f(m.quat), f(m.opacity), f(m.rgb), f(m.sem), gi)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    def tensors(self):
        return (self.xyz, self.scale, self.quat, self.opacity, self.rgb, self.sem)

    def c_struct(self) -> R.rogs_surfels:
        return R.surfels(self.xyz, self.scale, self.quat, self.opacity, self.rgb, self.sem, self.grid_index)


@dataclasses.dataclass
class Frame:
    """Output and state of one forward call over a fixed set of cameras."""
    cams: list
    cam_arr: object
    layout: R.rogs_state_layout
    out: torch.Tensor       # float[(3+C+1) * total_pixels]
    state: torch.Tensor     # uint8[layout.total_bytes]
    pix_base: List[int]
    generation: int = 0     # forwards run on this frame (its state belongs to the latest)
    owner: int = 0          # id() of the Renderer whose context laid the state out

    def view(self, v: int, C: int) -> torch.Tensor:
        """Planes [3+C+1, H, W] of view v."""
        c = self.cams[v]
        nch = 3 + C + 1
        b = nch * self.pix_base[v]
        return self.out[b: b + nch * c.width * c.height].view(nch, c.height, c.width)

    def state_section(self, name: str, dtype, count: int) -> torch.Tensor:
        off = getattr(self.layout, name)
        itemsize = torch.empty(0, dtype=dtype).element_size()
        return self.state[off: off + count * itemsize].view(dtype)


def _aligned_bytes(nbytes: int, device) -> torch.Tensor:
    t = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-t.data_ptr()) % 256
    return t[off: off + nbytes]


class Renderer:
    """Owns one librogs context (scratch, capacities, constants)."""

    def __init__(self, num_classes: int, record_capacity: int = 1 << 20, pair_capacity: int = 1 << 22,
                 tile=(16, 16), device="cuda", **consts):
        self.C = int(num_classes)
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.cfg = R.rogs_default_config(self.C, int(record_capacity), int(pair_capacity),
                                             tile_w=int(tile[0]), tile_h=int(tile[1]), **consts)
            self.ctx = R.rogs_create(self.cfg)

    def close(self):
        if getattr(self, "ctx", None):
            R.rogs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nch(self) -> int:
        return 3 + self.C + 1

    def reserve(self, n_surfels: int, n_views: int = None, cams: Sequence = None, training: bool = False):
        """Size the context's scratch up front (rogs_reserve): for n_surfels and
        n_views (or len(cams)); with training, also the backward's gradient rows
        and, given cams, the loss scratch for frames of those cameras.  Later
        calls then never allocate or synchronise (graph capture needs this)."""
        arr = R.cameras(cams) if cams is not None else None
        nv = len(cams) if cams is not None else int(n_views)
        R.rogs_reserve(self.ctx, n_surfels, nv, arr, training)

    def frame(self, cams: Sequence) -> Frame:
        arr = R.cameras(cams)
        L, elems = R.rogs_state_layout_of(self.ctx, arr, len(cams))
        out = torch.empty(elems, dtype=torch.float32, device=self.device)
        state = _aligned_bytes(int(L.total_bytes), self.device)
        pix, acc = [], 0
        for c in cams:
            pix.append(acc)
            acc += c.width * c.height
        return Frame(list(cams), arr, L, out, state, pix, owner=id(self))

    def _own(self, frame: Frame) -> Frame:
        # the state's section offsets follow this context's capacities: a frame
        # laid out by another context may be too small for them
        if frame.owner != id(self):
            raise ValueError("frame was made by another Renderer; make it with this renderer's frame()")
        return frame

    # -- the C-ABI calls --------------------------------------------------

    def forward(self, m: SurfelTensors, frame: Frame, exposure: torch.Tensor, stream=None) -> Frame:
        self._own(frame)
        frame.generation += 1
        R.rogs_render_fwd(self.ctx, m.c_struct(), frame.cam_arr, len(frame.cams), exposure, frame.out,
                          frame.state, stream)
        return frame

    def counts(self, frame: Frame, stream=None, check=True) -> R.rogs_counts:
        self._own(frame)
        return R.rogs_state_counts(self.ctx, frame.state, stream, check=check)

    def loss(self, frame: Frame, tgt_rgb, label, mask, lambda_c=1.0, lambda_s=0.06, loss=None, grad_out=None,
             stream=None):
        """Masked L1 + CE loss and dL/dout (rogs_loss).  Targets in the output
        pixel order: float32 colour planes with int32 labels, or uint8 colour
        planes (value / 255) with uint8 labels (rogs_loss_u8); uint8 mask."""
        self._own(frame)
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=self.device)
        if grad_out is None:
            grad_out = torch.empty_like(frame.out)
        R.rogs_loss(self.ctx, frame.cam_arr, len(frame.cams), frame.out, tgt_rgb, label, mask, lambda_c, lambda_s,
                    loss, grad_out, stream)
        return loss, grad_out

    def backward(self, m: SurfelTensors, frame: Frame, exposure: torch.Tensor, grad_out: torch.Tensor,
                 grads: Optional[dict] = None, stream=None) -> dict:
        self._own(frame)
        if grads is None:
            grads = zero_grads(m, exposure)
        R.rogs_render_bwd(self.ctx, m.c_struct(), frame.cam_arr, len(frame.cams), exposure, frame.state,
                          grad_out.contiguous(), self.grads_struct(grads), stream)
        return grads

    def grads_struct(self, grads: dict) -> R.rogs_grads:
        g = R.rogs_grads()
        for k in ("xyz", "scale", "quat", "opacity", "rgb", "sem", "exposure"):
            t = grads.get(k)
            setattr(g, k, t.data_ptr() if t is not None and t.numel() else None)
        return g

    def train_step(self, m: SurfelTensors, frame: Frame, exposure: torch.Tensor, tgt_rgb, label, mask,
                   loss: torch.Tensor, grads: dict, lambda_c=1.0, lambda_s=0.06, stream=None, lambda_smooth=0.0):
        """Forward, masked L1 + CE loss and backward with the loss fused into the
        backward kernel (rogs_train_step), plus lambda_smooth L_smooth when
        nonzero; gradients are added into `grads`.  Targets as in loss():
        uint8 colour and labels take rogs_train_step_u8."""
        self._own(frame)
        frame.generation += 1
        R.rogs_train_step(self.ctx, m.c_struct(), frame.cam_arr, len(frame.cams), exposure, frame.out, frame.state,
                          tgt_rgb, label, mask, lambda_c, lambda_s, loss, self.grads_struct(grads), stream,
                          lambda_smooth)

    def train_graph(self, m: SurfelTensors, frame: Frame, exposure: torch.Tensor, tgt_rgb, label, mask,
                    loss: torch.Tensor, grads: dict, lambda_c=1.0, lambda_s=0.06, stream=None,
                    lambda_smooth=0.0) -> "Graph":
        """Capture rogs_train_step of `frame` into a CUDA graph (all pointers
        fixed; `stream` must be a non-default stream)."""
        self._own(frame)
        g = R.rogs_train_graph_create(self.ctx, m.c_struct(), frame.cam_arr, len(frame.cams), exposure, frame.out,
                                      frame.state, tgt_rgb, label, mask, lambda_c, lambda_s, loss,
                                      self.grads_struct(grads), stream, lambda_smooth)
        return Graph(g, keep=(m, frame, exposure, tgt_rgb, label, mask, loss, grads))

    def bev_export(self, m: SurfelTensors, exposure: torch.Tensor, x0, y1, res, width, height, chunk=2000,
                   batch=4, cam_z=100.0, exposure_idx=0, stream=None) -> torch.Tensor:
        """Chunked BEV export (rogs_bev_export): [3 + C + 1, height, width] planes
        of the ground rectangle whose top-left corner is (x0, y1)."""
        image = torch.empty((3 + self.C + 1, height, width), device=m.xyz.device)
        R.rogs_bev_export(self.ctx, m.c_struct(), exposure, exposure_idx, x0, y1, res, cam_z, width, height, chunk,
                          batch, image, stream)
        return image

    def elev_targets(self, m: SurfelTensors, points: torch.Tensor, radius=0.1, stream=None) -> torch.Tensor:
        """LiDAR elevation targets zbar [n] (NaN where no point is within radius)."""
        zt = torch.empty(m.n, device=m.xyz.device)
        R.rogs_elev_targets(self.ctx, m.c_struct(), points, radius, zt, stream)
        return zt

    def elev_loss(self, m: SurfelTensors, z_target, lambda_z, loss, grad_xyz=None, stream=None):
        """loss[0] += lambda_z L_z; lambda_z dL/dz added into grad_xyz[:, 2]."""
        R.rogs_elev_loss(self.ctx, m.c_struct(), z_target, lambda_z, loss, grad_xyz, stream)
        return loss

    def smooth_loss(self, m: SurfelTensors, lambda_smooth=0.003, loss=None, grad_xyz=None, stream=None):
        """lambda * L_smooth over the grid index map (rogs_smooth_loss); the
        gradient is added into grad_xyz[:, 2] when given."""
        loss = torch.empty(1, device=m.xyz.device) if loss is None else loss
        R.rogs_smooth_loss(self.ctx, m.c_struct(), lambda_smooth, loss, grad_xyz, stream)
        return loss

    def render_graph(self, m: SurfelTensors, frame: Frame, exposure: torch.Tensor, stream=None) -> "Graph":
        self._own(frame)
        g = R.rogs_render_graph_create(self.ctx, m.c_struct(), frame.cam_arr, len(frame.cams), exposure, frame.out,
                                       frame.state, stream)
        return Graph(g, keep=(m, frame, exposure))

    def init_from_poses(self, grid_xy: torch.Tensor, poses: np.ndarray, exact_plane=True, stream=None):
        n = grid_xy.shape[0]
        z = torch.empty(n, dtype=torch.float32, device=self.device)
        q = torch.empty(n, 4, dtype=torch.float32, device=self.device)
        near = torch.empty(n, dtype=torch.int32, device=self.device)
        R.rogs_init_from_poses(self.ctx, grid_xy.contiguous(), poses, exact_plane, z, q, near, stream)
        return z, q, near

    def sort_pairs(self, keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32, stream=None):
        ko = torch.empty_like(keys)
        vo = torch.empty_like(vals)
        R.rogs_sort_pairs(self.ctx, keys, vals, key_bits, ko, vo, stream)
        return ko, vo


class Graph:
    """An executable CUDA graph captured by librogs; keeps its buffers alive."""

    def __init__(self, handle, keep=()):
        self.handle = handle
        self._keep = keep

    def launch(self, stream=None):
        R.rogs_graph_launch(self.handle, stream)

    def close(self):
        if self.handle:
            R.rogs_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zero_grads(m: SurfelTensors, exposure: torch.Tensor) -> dict:
    return dict(xyz=torch.zeros_like(m.xyz), scale=torch.zeros_like(m.scale), quat=torch.zeros_like(m.quat),
                opacity=torch.zeros_like(m.opacity), rgb=torch.zeros_like(m.rgb), sem=torch.zeros_like(m.sem),
                exposure=torch.zeros_like(exposure))


def targets_to_device(targets, device="cuda"):
    """Per-view planar targets -> flat device tensors in the output pixel order."""
    # planar per view: [3][pixels of view] blocks, view after view
    rgb = torch.cat([torch.as_tensor(np.ascontiguousarray(t, np.float32)).reshape(-1) for t in targets.rgb]).to(device)
    label = torch.cat([torch.as_tensor(np.ascontiguousarray(l, np.int32)).reshape(-1) for l in targets.label]).to(device)
    mask = torch.cat([torch.as_tensor(np.ascontiguousarray(k, np.uint8)).reshape(-1) for k in targets.mask]).to(device)
    return rgb.contiguous(), label.contiguous(), mask.contiguous()


class RenderFunction(torch.autograd.Function):
    """out = render(surfels, exposure); backward via rogs_render_bwd.

    The compositing state the backward recomputes from (records, tile lists,
    final transmittance and last contributor per pixel) lives in the frame, so
    the backward refuses to run if the frame was rendered again after this
    forward (its state would belong to the later forward).  The backward runs
    on the stream autograd gives it, after the forward's stream."""

    @staticmethod
    def forward(ctx, renderer: Renderer, frame: Frame, xyz, scale, quat, opacity, rgb, sem, exposure):
        m = SurfelTensors(xyz.detach(), scale.detach(), quat.detach(), opacity.detach(), rgb.detach(), sem.detach())
        stream = torch.cuda.current_stream(frame.out.device)
        renderer.forward(m, frame, exposure.detach(), stream)
        ctx.renderer, ctx.frame, ctx.m, ctx.exposure = renderer, frame, m, exposure.detach()
        ctx.generation, ctx.stream = frame.generation, stream
        return frame.out.clone()

    @staticmethod
    def backward(ctx, grad_out):
        if ctx.frame.generation != ctx.generation:
            raise RuntimeError("the frame was rendered again after this forward; render each graph's forward into "
                               "its own frame (render(..., frame=None)) before calling backward")
        stream = torch.cuda.current_stream(grad_out.device)
        if stream != ctx.stream:
            stream.wait_stream(ctx.stream)
        g = ctx.renderer.backward(ctx.m, ctx.frame, ctx.exposure, grad_out.contiguous(), stream=stream)
        return (None, None, g["xyz"], g["scale"], g["quat"], g["opacity"], g["rgb"], g["sem"], g["exposure"])


def render(renderer: Renderer, cams, xyz, scale, quat, opacity, rgb, sem, exposure, frame: Frame = None):
    """Differentiable render of `cams`; returns the flat output planes (view v
    at [(3+C+1) pix_base[v], ...), planes rgb, C logits, depth) and the frame."""
    frame = renderer.frame(cams) if frame is None else frame
    return RenderFunction.apply(renderer, frame, xyz, scale, quat, opacity, rgb, sem, exposure), frame


# Sec. 4.2 learning rates; z's rate is Z_LR_RANGE times the scene size,
# falling from the first value to the second over the training steps
PAPER_LR = {"opacity": 1e-4, "scale": 1e-4, "quat": 1e-4, "rgb": 0.008, "sem": 0.1, "exposure": 0.001}
Z_LR_RANGE = (1.6e-4, 1.6e-6)


class Adam:
    """Adam state (m, v) for a SurfelTensors + exposure tensor and one fused
    step over all of them (rogs_adam_step): z only of the positions (its rate
    decays inside the library from scene_size x 1.6e-4 to scene_size x 1.6e-6
    over total_steps; x and y gradients are cleared, not learnt), then
    opacity, scale, quat, rgb, sem, exposure with the paper's rates."""

    def __init__(self, renderer, m: SurfelTensors, exposure: torch.Tensor, scene_size: float, total_steps: int,
                 lr=None):
        self.r, self.m, self.exposure = renderer, m, exposure
        self.lr = dict(PAPER_LR if lr is None else lr)
        self.scene_size, self.total_steps = float(scene_size), int(total_steps)
        self.t = 0
        sizes = {"z": m.n, "opacity": m.opacity.numel(), "scale": m.scale.numel(), "quat": m.quat.numel(),
                 "rgb": m.rgb.numel(), "sem": m.sem.numel(), "exposure": exposure.numel()}
        self.state = {k: (torch.zeros(n, device=m.xyz.device), torch.zeros(n, device=m.xyz.device))
                      for k, n in sizes.items()}

    def step(self, grads: dict, zero_grad=True, stream=None):
        self.t += 1
        m = self.m
        groups = []
        mv = self.state
        z0, z1 = (self.scene_size * r for r in Z_LR_RANGE)
        groups.append((m.xyz[:, 2], grads["xyz"][:, 2], *mv["z"], m.n, 3, z0, z1, self.total_steps, 2))
        for k in ("opacity", "scale", "quat", "rgb", "sem"):
            p = getattr(m, k)
            if p.numel():
                groups.append((p, grads[k], *mv[k], p.numel(), 1, self.lr[k]))
        groups.append((self.exposure, grads["exposure"], *mv["exposure"], self.exposure.numel(), 1,
                       self.lr["exposure"]))
        R.rogs_adam_step(self.r.ctx, groups, self.t, zero_grad=zero_grad, stream=stream)
