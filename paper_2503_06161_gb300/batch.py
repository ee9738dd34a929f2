"""Batched rendering: many (time, camera, resolution) views of one deforming
scene rendered forward and backward in a single CUDA-graph launch, with the
parameter gradients summed over the views (the multi-view form of the pass).

Views run one after another on one stream and share one workspace; each view
uses the tile shape the autotuner picked for its resolution (the rendered
result does not depend on the tile shape: inclusion is per pixel).  The
first view overwrites the gradient buffers and the others add to them, so
the sum over views is formed in a fixed order (bitwise reproducible).

    br = BatchRenderer(scene, deform, [(cam0, t0), (cam1, t1), ...], targets)
    br.capture()          # records every launch of one batch into a CUDA graph
    br.replay()           # one graph launch: all views, forward + backward
"""
from __future__ import annotations

import dataclasses
import statistics

import torch

from . import _lib
from .raster import DeformField, GaussianScene, Rasterizer

TILE_SHAPES = ((16, 16), (32, 8), (8, 32))


class Autotuner:
    """Picks, per (width, height, P, D, storage), the tile shape with the
    fastest forward + backward, timed with CUDA events on the real scene.
    Results are cached for the life of the object."""

    def __init__(self, shapes=TILE_SHAPES, reps: int = 3):
        self.shapes, self.reps = tuple(shapes), int(reps)
        self.cache: dict = {}
        self.timings: dict = {}

    def pick(self, scene: GaussianScene, deform, cam, t, max_dups, workspace, grads, g_rgb, g_feat) -> tuple:
        key = (cam.width, cam.height, scene.P, scene.D, str(scene.feat.dtype))
        if key in self.cache:
            return self.cache[key]
        best, best_ms, times = None, float("inf"), {}
        for shape in self.shapes:
            if cam.width < shape[0] and cam.height < shape[1]:
                continue
            r = Rasterizer(scene.P, scene.D, cam.width, cam.height, tile=shape, max_dups=max_dups,
                           device=workspace.device, auto_grow=False, workspace=workspace)
            ms = []
            for k in range(self.reps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                r.forward(scene, cam, deform, t)
                r.backward(scene, cam, deform, t, g_rgb, None, None, g_feat, grads=grads)
                e1.record()
                torch.cuda.synchronize()
                if k:
                    ms.append(e0.elapsed_time(e1))
            times[shape] = statistics.median(ms)
            if times[shape] < best_ms:
                best, best_ms = shape, times[shape]
        self.cache[key] = best
        self.timings[key] = times
        return best


@dataclasses.dataclass
class View:
    cam: _lib.fe_camera
    t: float
    tgt_rgb: torch.Tensor    # [3,H,W]
    tgt_feat: torch.Tensor   # [H*W, D]


class BatchRenderer:
    def __init__(self, scene: GaussianScene, deform: DeformField | None, views: list, autotuner: Autotuner | None,
                 capacity_margin: float = 1.5, device="cuda"):
        self.scene, self.deform, self.views = scene, deform, list(views)
        P, D = scene.P, scene.D
        self.device = torch.device(device)
        kw = dict(dtype=torch.float32, device=self.device)
        self.grads = dict(means=torch.zeros(P, 3, **kw), log_scales=torch.zeros(P, 3, **kw),
                          quats=torch.zeros(P, 4, **kw), opacity_logits=torch.zeros(P, **kw),
                          sh=torch.zeros(P, 16, 3, **kw), feat=torch.zeros(P, D, **kw))
        # Capacity of each view's (Gaussian, tile) list from a probe forward;
        # one workspace, sized for the largest view, serves every view.
        caps, sizes = [], []
        for v in self.views:
            probe = Rasterizer(P, D, v.cam.width, v.cam.height, max_dups=64 * P + 4096, forward_only=True,
                               device=self.device)
            probe.forward(scene, v.cam, deform, v.t)
            caps.append(int(probe.stats()["num_dups"] * capacity_margin) + 4096)
            del probe
        for v, cap in zip(self.views, caps):
            sizes.append(max(Rasterizer.workspace_bytes(P, D, v.cam.width, v.cam.height, tile=s, max_dups=cap)
                             for s in TILE_SHAPES))
        torch.cuda.empty_cache()
        self.workspace = torch.empty(max(sizes), dtype=torch.uint8, device=self.device)
        self.bufs = []
        for v in self.views:
            H, W = v.cam.height, v.cam.width
            self.bufs.append(dict(out=(torch.empty(3, H, W, **kw), torch.empty(H, W, **kw), torch.empty(H, W, **kw),
                                       torch.empty(H * W, D, **kw)),
                                  g_rgb=torch.empty(3, H, W, **kw), g_feat=torch.empty(H * W, D, **kw)))
        self.losses = torch.zeros(len(self.views), 2, **kw)
        self.scratch = torch.empty(len(self.views), 2, 1024, **kw)
        # Device error bits of each view (the shared workspace's header is
        # cleared by every forward), copied out after each view.
        self.errs = torch.zeros(len(self.views), dtype=torch.int32, device=self.device)
        for b in self.bufs:  # upstream gradients for the tuning runs
            b["g_rgb"].fill_(1e-3)
            b["g_feat"].fill_(1e-3)
        # Tile shape per view (autotuned per resolution, else 16x16).
        self.rasts = []
        for k, (v, cap) in enumerate(zip(self.views, caps)):
            shape = (16, 16)
            if autotuner is not None:
                b = self.bufs[k]
                shape = autotuner.pick(scene, deform, v.cam, v.t, cap, self.workspace, self.grads, b["g_rgb"],
                                       b["g_feat"])
            self.rasts.append(Rasterizer(P, D, v.cam.width, v.cam.height, tile=shape, max_dups=cap,
                                         device=self.device, auto_grow=False, accumulate=k > 0,
                                         workspace=self.workspace))
        self.graph = None

    @property
    def tile_shapes(self):
        return [r.tile for r in self.rasts]

    def run(self):
        """All views: forward, L1 losses (RGB and features), backward; the
        gradients are summed into self.grads."""
        for k, (v, r, b) in enumerate(zip(self.views, self.rasts, self.bufs)):
            HW = v.cam.width * v.cam.height
            r.forward(self.scene, v.cam, self.deform, v.t, out=b["out"])
            _lib.fe_l1_loss_grad(b["out"][0], v.tgt_rgb, HW, b["g_rgb"], self.losses[k, 0:1], self.scratch[k, 0])
            _lib.fe_l1_loss_grad(b["out"][3], v.tgt_feat, HW, b["g_feat"], self.losses[k, 1:2], self.scratch[k, 1])
            r.backward(self.scene, v.cam, self.deform, v.t, b["g_rgb"], None, None, b["g_feat"], grads=self.grads)
            self.errs[k:k + 1].copy_(self.workspace[:4].view(torch.int32))

    def capture(self):
        """Record one batch into a CUDA graph (after one eager warm-up run)."""
        self.run()
        torch.cuda.synchronize()
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def device_errors(self) -> int:
        """OR over the views of the device error bits of the last run
        (synchronises): 1 = a view's list overflowed its capacity."""
        e = 0
        for x in self.errs.cpu().tolist():
            e |= int(x)
        return e
