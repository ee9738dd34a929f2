"""The full FST deformation module (Sec. 3.2, Eq. 4-6; Appendix A) on the
device: multi-resolution HexPlane, decoder MLP F_out, four geometric
branches and the semantic updater F_feat.  Every step runs in the library's
kernels (fe_fst_forward / fe_fst_backward / fe_fst_tv); this module owns the
device buffers and marshals the calls.

It wraps the renderer: ``forward`` writes the deformed Gaussians G_t
(Eq. 6) into a GaussianScene that a static render consumes, and
``backward`` turns that render's parameter gradients into the gradients of
the canonical Gaussians, the planes and every MLP weight.

    fst = FSTDeform(planes, mlp, levels=4, rs=64, rt=100, D=32, bbox=..., P=P)
    scene_t = fst.forward(scene, t)
    rast.forward(scene_t, cam, None, t); rast.backward(..., grads=g)
    fst.backward(scene, t, g)          # g["means"] gains the HexPlane path
"""
from __future__ import annotations

import torch

from . import _lib
from .raster import GaussianScene


class FSTDeform:
    def __init__(self, planes: torch.Tensor, mlp: torch.Tensor, levels: int, rs: int, rt: int, D: int, bbox_min,
                 bbox_max, P: int, with_backward: bool = True, device="cuda", exact_planes: bool = False):
        """exact_planes: plane gradients as exact fixed-point sums (bitwise
        reproducible, about twice the reverse's time) instead of float
        atomics."""
        self.levels, self.rs, self.rt, self.D, self.P = int(levels), int(rs), int(rt), int(D), int(P)
        self.exact_planes = bool(exact_planes)
        dev = torch.device(device)
        self.planes = planes.to(dev, torch.float32).contiguous()
        self.mlp = mlp.to(dev, torch.float32).contiguous()
        if self.planes.numel() != _lib.fe_fst_plane_floats(levels, rs, rt):
            raise ValueError("plane array size does not match (levels, rs, rt)")
        if self.mlp.numel() != _lib.fe_fst_mlp_floats(levels, D):
            raise ValueError("MLP array size does not match (levels, D)")
        self.bbox_min, self.bbox_max = tuple(float(x) for x in bbox_min), tuple(float(x) for x in bbox_max)
        self.with_backward = bool(with_backward)
        self.workspace = torch.empty(_lib.fe_fst_workspace_size(P, levels, rs, rt, D, self._wb()),
                                     dtype=torch.uint8, device=dev)
        self.d_planes = torch.zeros_like(self.planes)
        self.d_mlp = torch.zeros_like(self.mlp)
        self._out = None

    def resize(self, P: int):
        """Workspace for a new Gaussian count (after densification)."""
        self.P = int(P)
        self.workspace = None
        self.workspace = torch.empty(_lib.fe_fst_workspace_size(self.P, self.levels, self.rs, self.rt, self.D,
                                                                self._wb()),
                                     dtype=torch.uint8, device=self.planes.device)
        self._out = None

    @classmethod
    def from_numpy(cls, planes, mlp, levels, rs, rt, D, bbox_min, bbox_max, P, device="cuda", **kw):
        return cls(torch.as_tensor(planes), torch.as_tensor(mlp), levels, rs, rt, D, bbox_min, bbox_max, P,
                   device=device, **kw)

    def _wb(self) -> int:
        return (2 if self.exact_planes else 1) if self.with_backward else 0

    def struct(self) -> _lib.fe_fst:
        return _lib.make_fst(self.levels, self.rs, self.rt, self.D, self.planes, self.mlp, self.bbox_min,
                             self.bbox_max, self.exact_planes)

    def _buffers(self, scene: GaussianScene):
        key = (scene.P, scene.feat.dtype, scene.means.device)
        if self._out is None or self._out[0] != key:
            P, dev = scene.P, scene.means.device
            f = dict(dtype=torch.float32, device=dev)
            self._out = (key, dict(means=torch.empty(P, 3, **f), quats=torch.empty(P, 4, **f),
                                   log_scales=torch.empty(P, 3, **f), opacity_logits=torch.empty(P, **f),
                                   feat=torch.empty(P, self.D, dtype=scene.feat.dtype, device=dev)))
        return self._out[1]

    def forward(self, scene: GaussianScene, t: float, stream=None) -> GaussianScene:
        """G_t: the deformed Gaussians (SH shared with the canonical scene)."""
        if scene.P != self.P or scene.D != self.D:
            raise ValueError("scene size does not match the module")
        o = self._buffers(scene)
        _lib.fe_fst_forward(self.struct(), scene.P, scene.means, scene.quats, scene.log_scales,
                            scene.opacity_logits, scene.feat, t, o["means"], o["quats"], o["log_scales"],
                            o["opacity_logits"], o["feat"], self.workspace, self.with_backward, stream)
        return GaussianScene(o["means"], o["log_scales"], o["quats"], o["opacity_logits"], scene.sh, o["feat"],
                             scene.sh_degree)

    def backward(self, scene: GaussianScene, t: float, grads: dict, stream=None):
        """Reverse of the last forward.  grads: the renderer's gradients of
        the deformed Gaussians (means, quats, log_scales, opacity_logits,
        feat, float32); they are also those of the canonical ones, except
        grads["means"], which gains the path through the HexPlane
        coordinates (in place).  Fills self.d_planes and self.d_mlp."""
        if not self.with_backward:
            raise RuntimeError("module built without backward state")
        _lib.fe_fst_backward(self.struct(), scene.P, scene.means, t, grads["means"], grads["quats"],
                             grads["log_scales"], grads["opacity_logits"], grads["feat"], grads["means"],
                             self.d_planes, self.d_mlp, self.workspace, stream)

    def tv(self, weight: float, loss: torch.Tensor, scratch: torch.Tensor, stream=None):
        """Adds weight * dL_TV/dplanes to self.d_planes; loss (one device
        float) = weight * L_TV (Eq. 11)."""
        _lib.fe_fst_tv(self.struct(), weight, loss, self.d_planes, scratch, stream)
