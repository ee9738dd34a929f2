"""Torch-facing API over the C ABI: device tensors in, device tensors out.

PyTorch supplies device memory, the CUDA stream and autograd plumbing; every
step of the pass runs in the library's kernels.

    scene = GaussianScene.from_numpy(synth_scene, device="cuda")
    cam = camera_struct(synth_camera)
    rast = Rasterizer(scene.P, scene.D, cam.width, cam.height)
    rgb, depth, alpha, feat = render(rast, scene, cam, deform=None, t=0.0)
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _lib


@dataclasses.dataclass
class GaussianScene:
    """Canonical Gaussians on the device (Sec. 3.1; feature z of Sec. 3.2)."""
    means: torch.Tensor           # [P,3] f32
    log_scales: torch.Tensor      # [P,3] f32
    quats: torch.Tensor           # [P,4] f32 (w,x,y,z)
    opacity_logits: torch.Tensor  # [P] f32
    sh: torch.Tensor              # [P,16,3] f32 or bf16
    feat: torch.Tensor            # [P,D] f32 or bf16
    sh_degree: int = 3

    @property
    def P(self) -> int:
        return int(self.means.shape[0])

    @property
    def D(self) -> int:
        return int(self.feat.shape[1])

    @classmethod
    def from_numpy(cls, s, device="cuda", bf16: bool = False) -> "GaussianScene":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)
        sh = f(np.asarray(s.sh).reshape(s.P, 16, 3))
        feat = f(s.feat)
        if bf16:
            sh = sh.to(torch.bfloat16)
            feat = feat.to(torch.bfloat16)
        return cls(f(s.means), f(s.log_scales), f(s.quats), f(s.opacity_logits), sh, feat, int(s.sh_degree))

    def params(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logits, self.sh, self.feat]

    def struct(self) -> _lib.fe_gaussians:
        return _lib.make_gaussians(self.means, self.log_scales, self.quats, self.opacity_logits, self.sh, self.feat,
                                   self.sh_degree)


@dataclasses.dataclass
class DeformField:
    """HexPlane + MLP deformation field on the device (Sec. 3.2, Eq. 4-6)."""
    planes: torch.Tensor   # [6,R,R,C]
    w1: torch.Tensor
    b1: torch.Tensor
    w2: torch.Tensor
    b2: torch.Tensor
    wh: torch.Tensor
    bh: torch.Tensor
    bbox_min: tuple
    bbox_max: tuple
    noise: torch.Tensor | None = None
    noise_scale: float = 0.01

    @classmethod
    def from_numpy(cls, d, device="cuda") -> "DeformField":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device=device)
        return cls(f(d.planes), f(d.w1), f(d.b1), f(d.w2), f(d.b2), f(d.wh), f(d.bh),
                   tuple(float(x) for x in d.bbox_min), tuple(float(x) for x in d.bbox_max),
                   f(d.noise) if d.noise is not None else None, float(d.noise_scale))

    def struct(self) -> _lib.fe_deform:
        return _lib.make_deform(self.planes, self.w1, self.b1, self.w2, self.b2, self.wh, self.bh, self.bbox_min,
                                self.bbox_max, self.noise, self.noise_scale)


def camera_struct(cam) -> _lib.fe_camera:
    """fe_camera from an object with width, height, fx, fy, cx, cy,
    world_to_cam [4,4], campos [3], znear."""
    return _lib.make_camera(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy,
                            np.asarray(cam.world_to_cam, np.float32).reshape(16),
                            np.asarray(cam.campos, np.float32).reshape(3), cam.znear)


class Rasterizer:
    """Owns the device workspace for one (P, D, width, height, options)
    shape.  One forward may be outstanding at a time: its backward must use
    the same Rasterizer before the next forward."""

    def __init__(self, P: int, D: int, width: int, height: int, tile=(16, 16), bg=(0.0, 0.0, 0.0),
                 max_dups: int = 0, forward_only: bool = False, device="cuda", auto_grow: bool | None = None,
                 accumulate: bool = False, workspace: torch.Tensor | None = None, fwd_batch: int = 0,
                 wait_polls: int = 0):
        """accumulate: backward adds to the gradient buffers instead of
        overwriting them.  workspace: optional uint8 device tensor to use
        (e.g. one buffer shared by views that are rendered one after the
        other); it must hold workspace_bytes(...).  fwd_batch: Gaussians per
        staged batch of the compositing forward (0 = default).  wait_polls:
        test hook of the staging-wait bound (fe_opts.wait_polls)."""
        self.P, self.D, self.width, self.height = int(P), int(D), int(width), int(height)
        self.tile, self.bg, self.forward_only = tuple(tile), tuple(bg), bool(forward_only)
        self.accumulate = bool(accumulate)
        self.fwd_batch, self.wait_polls = int(fwd_batch), int(wait_polls)
        self.device = torch.device(device)
        # Without an explicit capacity, the FIRST forward reads the list size
        # back (one host sync) and grows the list to 1.5x what it needed;
        # later forwards read nothing back.  An overflow is still recorded on
        # the device (the overflowing tiles are left empty): check() reads it.
        self.auto_grow = (max_dups == 0) if auto_grow is None else bool(auto_grow)
        self._sized = False
        self._alloc(int(max_dups), workspace)

    @staticmethod
    def workspace_bytes(P, D, width, height, tile=(16, 16), max_dups=0, forward_only=False) -> int:
        return _lib.fe_workspace_size(int(P), int(D), int(width), int(height),
                                      _lib.make_opts(tuple(tile), (0.0, 0.0, 0.0), int(max_dups), forward_only))

    def _alloc(self, max_dups: int, workspace: torch.Tensor | None = None):
        self.opts = _lib.make_opts(self.tile, self.bg, max_dups, self.forward_only, self.accumulate, self.fwd_batch,
                                   self.wait_polls)
        self.nbytes = _lib.fe_workspace_size(self.P, self.D, self.width, self.height, self.opts)
        if workspace is not None:
            if workspace.numel() * workspace.element_size() < self.nbytes or workspace.dtype != torch.uint8:
                raise ValueError(f"shared workspace too small: {self.nbytes} bytes needed")
            self.workspace = workspace[:self.nbytes]
            return
        self.workspace = None
        self.workspace = torch.empty(self.nbytes, dtype=torch.uint8, device=self.device)

    @property
    def capacity(self) -> int:
        return int(self.opts.max_dups) if self.opts.max_dups > 0 else 16 * self.P + 4096

    def forward(self, scene: GaussianScene, cam: _lib.fe_camera, deform: DeformField | None = None, t: float = 0.0,
                out=None, feat_bf16=None):
        """(rgb, depth, alpha, feat); feat_bf16: optional [H*W, D] bf16 tensor
        that also receives the feature map rounded to bf16 (decoder input)."""
        H, W, D = self.height, self.width, self.D
        if out is None:
            kw = dict(dtype=torch.float32, device=self.device)
            out = (torch.empty(3, H, W, **kw), torch.empty(H, W, **kw), torch.empty(H, W, **kw),
                   torch.empty(H * W, D, **kw))
        rgb, depth, alpha, feat = out
        for _ in range(4):
            _lib.fe_render_forward(scene.struct(), deform.struct() if deform is not None else None, cam, t,
                                   self.opts, self.workspace, rgb, depth, alpha, feat, feat_bf16=feat_bf16)
            if not self.auto_grow or self._sized:
                break
            st = self.stats(raise_on_error=False)
            # Sized once the list fits with a 1.5x margin for later frames;
            # otherwise grow and render again (the state the backward reads
            # must be in the workspace that stays).
            if not (st["device_errors"] & 1) and st["num_dups"] * 3 <= 2 * self.capacity:
                self._sized = True
                break
            self._alloc(int(st["num_dups"] * 1.5) + 4096)
        return rgb, depth, alpha, feat

    def check(self):
        """Raises if the last forward overflowed its list or hit another
        device-side error (synchronises the stream)."""
        self.stats(raise_on_error=True)

    def backward(self, scene: GaussianScene, cam: _lib.fe_camera, deform: DeformField | None, t: float,
                 g_rgb=None, g_depth=None, g_alpha=None, g_feat=None, grads=None):
        P, D = self.P, self.D
        if grads is None:
            kw = dict(dtype=torch.float32, device=self.device)
            grads = dict(means=torch.empty(P, 3, **kw), log_scales=torch.empty(P, 3, **kw),
                         quats=torch.empty(P, 4, **kw), opacity_logits=torch.empty(P, **kw),
                         sh=torch.empty(P, 16, 3, **kw), feat=torch.empty(P, D, **kw))
        c = lambda x: None if x is None else x.contiguous()
        _lib.fe_render_backward(scene.struct(), deform.struct() if deform is not None else None, cam, t, self.opts,
                                self.workspace, c(g_rgb), c(g_depth), c(g_alpha), c(g_feat), grads["means"],
                                grads["log_scales"], grads["quats"], grads["opacity_logits"], grads["sh"],
                                grads["feat"])
        return grads

    def stats(self, raise_on_error: bool = True) -> dict:
        return _lib.fe_read_stats(self.workspace, self.P, self.D, self.width, self.height, self.opts,
                                  raise_on_error=raise_on_error)

    def dump(self) -> dict:
        """Forward state for parity tests (synchronous)."""
        st = self.stats(raise_on_error=False)
        K = int(min(st["num_dups"], st["capacity"]))
        dev = self.device
        P, HW = self.P, self.width * self.height
        tw, th = self.opts.tile_w, self.opts.tile_h
        ntiles = ((self.width + tw - 1) // tw) * ((self.height + th - 1) // th)
        o = dict(keys=torch.zeros(max(K, 1), dtype=torch.int64, device=dev),
                 gauss=torch.zeros(max(K, 1), dtype=torch.int32, device=dev),
                 ranges=torch.zeros(ntiles, 2, dtype=torch.int32, device=dev),
                 n_contrib=torch.zeros(HW, dtype=torch.int32, device=dev),
                 t_final=torch.zeros(HW, dtype=torch.float32, device=dev),
                 uv=torch.zeros(P, 2, device=dev), conic=torch.zeros(P, 3, device=dev),
                 opacity=torch.zeros(P, device=dev), depth=torch.zeros(P, device=dev),
                 rgb=torch.zeros(P, 3, device=dev), radius=torch.zeros(P, dtype=torch.int32, device=dev),
                 touched=torch.zeros(P, dtype=torch.int32, device=dev))
        # The dump only reads regions below the D-dependent part of the layout.
        _lib.fe_debug_dump(self.workspace, P, self.D, self.width, self.height, self.opts, **o)
        torch.cuda.synchronize(dev)
        o["keys"] = o["keys"][:K]
        o["gauss"] = o["gauss"][:K]
        o["K"] = K
        o["stats"] = st
        return o


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rast, scene_meta, cam, deform, t, means, log_scales, quats, opacity_logits, sh, feat):
        scene = GaussianScene(means, log_scales, quats, opacity_logits, sh, feat, scene_meta)
        rgb, depth, alpha, fmap = rast.forward(scene, cam, deform, t)
        ctx.rast, ctx.cam, ctx.deform, ctx.t, ctx.scene = rast, cam, deform, t, scene
        return rgb, depth, alpha, fmap

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha, g_feat):
        g = ctx.rast.backward(ctx.scene, ctx.cam, ctx.deform, ctx.t, g_rgb, g_depth, g_alpha, g_feat)
        sh_dtype, feat_dtype = ctx.scene.sh.dtype, ctx.scene.feat.dtype
        return (None, None, None, None, None, g["means"], g["log_scales"], g["quats"], g["opacity_logits"],
                g["sh"].to(sh_dtype), g["feat"].to(feat_dtype))


def render(rast: Rasterizer, scene: GaussianScene, cam: _lib.fe_camera, deform: DeformField | None = None,
           t: float = 0.0):
    """Differentiable render: (rgb [3,H,W], depth [H,W], alpha [H,W],
    feat [H*W,D]) with gradients to the scene's tensors."""
    return _RenderFn.apply(rast, scene.sh_degree, cam, deform, float(t), scene.means, scene.log_scales, scene.quats,
                           scene.opacity_logits, scene.sh, scene.feat)
