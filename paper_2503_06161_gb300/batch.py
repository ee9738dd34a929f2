"""Batched rendering: many (time, camera, resolution) views of one deforming
scene rendered forward and backward through the library's batched entry
points (fe_render_batch / fe_render_batch_backward), the parameter gradients
summed over the views.

Per view the per-Gaussian stages (deformation query, projection, colour,
binning) run one after another; the compositing of all views is ONE
persistent launch whose blocks take (view, tile) work items from a device
counter, and so is its reverse, so small views no longer leave the GPU half
empty.  Each view uses the tile shape the autotuner picked for its
resolution, and the whole batch the forward batch size (Gaussians per
shared-memory batch) it picked; neither changes an image (inclusion is per
pixel, the staging unit is not part of the arithmetic).  The batch step --
forward, the per-view L1 losses, reverse -- is captured into one CUDA graph
and replayed as one launch.

    br = BatchRenderer(scene, deform, views, Autotuner())
    br.capture()
    br.replay()
"""
from __future__ import annotations

import dataclasses
import statistics

import torch

from . import _lib
from .raster import DeformField, GaussianScene, Rasterizer

TILE_SHAPES = ((16, 16), (32, 8), (8, 32))
FWD_BATCHES = (32, 64, 128)
GRAD_SHAPES = (("means", (3,)), ("log_scales", (3,)), ("quats", (4,)), ("opacity_logits", ()), ("sh", (16, 3)))


def _time(fn, reps: int) -> float:
    ms = []
    for k in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        if k:
            ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


class Autotuner:
    """Picks, per (width, height, P, D, storage), the tile shape with the
    fastest forward + backward, and per batch the forward batch size,
    timed with CUDA events on the real scene.  Results are cached for the
    life of the object."""

    def __init__(self, shapes=TILE_SHAPES, fwd_batches=FWD_BATCHES, reps: int = 3):
        self.shapes, self.fwd_batches, self.reps = tuple(shapes), tuple(fwd_batches), int(reps)
        self.cache: dict = {}
        self.timings: dict = {}

    def pick_tile(self, scene: GaussianScene, deform, cam, t, max_dups, g_rgb, g_feat) -> tuple:
        key = (cam.width, cam.height, scene.P, scene.D, str(scene.feat.dtype))
        if key in self.cache:
            return self.cache[key]
        best, best_ms, times = (16, 16), float("inf"), {}
        for shape in self.shapes:
            if cam.width < shape[0] and cam.height < shape[1]:
                continue
            r = Rasterizer(scene.P, scene.D, cam.width, cam.height, tile=shape, max_dups=max_dups,
                           device=scene.means.device, auto_grow=False)

            def step():
                r.forward(scene, cam, deform, t)
                r.backward(scene, cam, deform, t, g_rgb, None, None, g_feat)

            times[shape] = _time(step, self.reps)
            if times[shape] < best_ms:
                best, best_ms = shape, times[shape]
            del r
        self.cache[key] = best
        self.timings[key] = times
        return best

    def pick_fwd_batch(self, renderer: "BatchRenderer") -> int:
        key = ("fwd_batch", tuple((v.cam.width, v.cam.height) for v in renderer.views), renderer.scene.P,
               renderer.scene.D, str(renderer.scene.feat.dtype))
        if key in self.cache:
            return self.cache[key]
        best, best_ms, times = 0, float("inf"), {}
        for B in self.fwd_batches:
            if B == 128 and renderer.scene.D > 64:
                continue
            renderer.set_fwd_batch(B)
            times[B] = _time(renderer.run, self.reps)
            if times[B] < best_ms:
                best, best_ms = B, times[B]
        self.cache[key] = best
        self.timings[key] = times
        return best


@dataclasses.dataclass
class View:
    cam: _lib.fe_camera
    t: float
    tgt_rgb: torch.Tensor    # [3,H,W]
    tgt_feat: torch.Tensor   # [H*W, D]


def _segments(P: int, D: int):
    """(name, shape, offset) of each gradient in one flat float32 buffer;
    every segment starts on a 16-byte boundary."""
    out, off = [], 0
    for name, shape in GRAD_SHAPES + (("feat", (D,)),):
        n = P
        for s in shape:
            n *= s
        out.append((name, shape, off))
        off += (n + 3) // 4 * 4
    return out, off


def _grad_views(flat: torch.Tensor, P: int, D: int) -> dict:
    """Named gradient tensors carved out of one flat float32 buffer."""
    segs, _ = _segments(P, D)
    out = {}
    for name, shape, off in segs:
        n = P
        for s in shape:
            n *= s
        out[name] = flat[off:off + n].view(P, *shape)
    return out


def grad_floats(P: int, D: int) -> int:
    return _segments(P, D)[1]


class BatchRenderer:
    """Owns the batch workspace, the per-view image and gradient buffers and
    the summed parameter gradients of one batch of views."""

    def __init__(self, scene: GaussianScene, deform: DeformField | None, views: list, autotuner: Autotuner | None,
                 capacity_margin: float = 1.5, fwd_batch: int = 0, tiles=None, device="cuda"):
        """tiles: optional tile shape per view (else autotuned, or 16x16
        without an autotuner); fwd_batch: 0 = autotuned (default size
        without an autotuner)."""
        if not 1 <= len(views) <= _lib.FE_MAX_VIEWS:
            raise ValueError(f"1..{_lib.FE_MAX_VIEWS} views per batch")
        self.scene, self.deform, self.views = scene, deform, list(views)
        P, D = scene.P, scene.D
        self.device = torch.device(device)
        kw = dict(dtype=torch.float32, device=self.device)
        self.flat = torch.zeros(grad_floats(P, D), **kw)
        self.grads = _grad_views(self.flat, P, D)
        self.bufs = []
        for v in self.views:
            H, W = v.cam.height, v.cam.width
            self.bufs.append(dict(out=(torch.empty(3, H, W, **kw), torch.empty(H, W, **kw), torch.empty(H, W, **kw),
                                       torch.empty(H * W, D, **kw)),
                                  g_rgb=torch.full((3, H, W), 1e-3, **kw), g_feat=torch.full((H * W, D), 1e-3, **kw)))
        # Capacity of each view's (Gaussian, tile) list from a probe forward.
        self.caps = []
        for v in self.views:
            probe = Rasterizer(P, D, v.cam.width, v.cam.height, max_dups=64 * P + 4096, forward_only=True,
                               device=self.device)
            probe.forward(scene, v.cam, deform, v.t)
            self.caps.append(int(probe.stats()["num_dups"] * capacity_margin) + 4096)
            del probe
        torch.cuda.empty_cache()
        if tiles is not None:
            self.tiles = [tuple(x) for x in tiles]
        elif autotuner is not None:
            self.tiles = [autotuner.pick_tile(scene, deform, v.cam, v.t, cap, b["g_rgb"], b["g_feat"])
                          for v, cap, b in zip(self.views, self.caps, self.bufs)]
        else:
            self.tiles = [(16, 16)] * len(self.views)
        self.losses = torch.zeros(len(self.views), 2, **kw)
        self.scratch = torch.empty(len(self.views), 2, 1024, **kw)
        self.fwd_batch = int(fwd_batch)
        self._build()
        if autotuner is not None and fwd_batch == 0:
            self.set_fwd_batch(autotuner.pick_fwd_batch(self))
        self.graph = None

    def _build(self, wait_polls: int = 0):
        opts = [_lib.make_opts(tile=shape, max_dups=cap, fwd_batch=self.fwd_batch, wait_polls=wait_polls)
                for shape, cap in zip(self.tiles, self.caps)]
        self.batch = _lib.make_batch([v.cam for v in self.views], [v.t for v in self.views], opts)
        nbytes = _lib.fe_batch_workspace_size(self.scene.P, self.scene.D, self.batch)
        if getattr(self, "workspace", None) is None or self.workspace.numel() < nbytes:
            self.workspace = None
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def set_fwd_batch(self, B: int):
        self.fwd_batch = int(B)
        self._build()
        self.graph = None

    def set_wait_polls(self, polls: int):
        """Test hook of the staging-wait bound (fe_opts.wait_polls)."""
        self._build(wait_polls=polls)
        self.graph = None

    @property
    def tile_shapes(self):
        return list(self.tiles)

    def view_workspace(self, k: int):
        """(single-view workspace slice, its fe_opts) of view k inside the
        batch workspace (a 256-byte header, then the views' workspaces)."""
        off = 256
        for j in range(k):
            off += _lib.fe_workspace_size(self.scene.P, self.scene.D, self.views[j].cam.width,
                                          self.views[j].cam.height, self.batch._opts[j])
        o = self.batch._opts[k]
        n = _lib.fe_workspace_size(self.scene.P, self.scene.D, self.views[k].cam.width, self.views[k].cam.height, o)
        return self.workspace[off:off + n], o

    def forward(self):
        g = self.scene.struct()
        d = self.deform.struct() if self.deform is not None else None
        _lib.fe_render_batch(g, d, self.batch, self.workspace, [b["out"] for b in self.bufs])

    def losses_and_grads(self):
        """Per view, the L1 losses of the rendered RGB and feature maps to the
        view's targets and their gradients (the upstream gradients)."""
        for k, (v, b) in enumerate(zip(self.views, self.bufs)):
            HW = v.cam.width * v.cam.height
            _lib.fe_l1_loss_grad(b["out"][0], v.tgt_rgb, HW, b["g_rgb"], self.losses[k, 0:1], self.scratch[k, 0])
            _lib.fe_l1_loss_grad(b["out"][3], v.tgt_feat, HW, b["g_feat"], self.losses[k, 1:2], self.scratch[k, 1])

    def backward(self):
        g = self.scene.struct()
        d = self.deform.struct() if self.deform is not None else None
        _lib.fe_render_batch_backward(g, d, self.batch, self.workspace,
                                      [(b["g_rgb"], None, None, b["g_feat"]) for b in self.bufs], self.grads)

    def run(self):
        """All views: forward, L1 losses (RGB and features), backward; the
        gradients are summed over the views into self.grads."""
        self.forward()
        self.losses_and_grads()
        self.backward()

    def capture(self):
        """Record one batch step into a CUDA graph (after one eager warm-up run)."""
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

    def stats(self, raise_on_error: bool = False):
        """(status, per-view statistics) of the last batch call (synchronises)."""
        return _lib.fe_batch_read_stats(self.workspace, self.scene.P, self.scene.D, self.batch,
                                        raise_on_error=raise_on_error)

    def device_errors(self) -> int:
        """OR over the views of the device error bits of the last run
        (synchronises): 1 = a list overflowed, 2 = a bounded wait gave up."""
        e = 0
        for st in self.stats()[1]:
            e |= int(st["device_errors"])
        return e
