"""Batched rendering: many (time, camera, resolution) views of one deforming
scene rendered forward and backward in a single CUDA-graph launch, with the
parameter gradients summed over the views (the multi-view form of the pass).

The views are dealt round-robin to S streams.  Each stream renders its views
one after another with its own workspace and its own gradient buffer (its
first view overwrites, the others add); the streams run concurrently, so the
launches of one view fill the GPU where another's leave it idle.  At the join
one kernel sums the S gradient buffers in stream order, so the result is
reproducible bit for bit.  Each view uses the tile shape the autotuner picked
for its resolution (the images do not depend on the tile shape: inclusion is
per pixel).  The whole batch -- fork, every view's launches, join, sum -- is
captured into one CUDA graph and replayed as one launch.

    br = BatchRenderer(scene, deform, views, Autotuner(), streams=4)
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
GRAD_SHAPES = (("means", (3,)), ("log_scales", (3,)), ("quats", (4,)), ("opacity_logits", ()), ("sh", (16, 3)))


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
    def __init__(self, scene: GaussianScene, deform: DeformField | None, views: list, autotuner: Autotuner | None,
                 streams: int = 4, capacity_margin: float = 1.5, device="cuda"):
        self.scene, self.deform, self.views = scene, deform, list(views)
        P, D = scene.P, scene.D
        self.device = torch.device(device)
        self.S = max(1, min(int(streams), len(self.views), 8))
        kw = dict(dtype=torch.float32, device=self.device)
        nflat = grad_floats(P, D)
        # Gradient buffer per stream; the batch's sum (stream 0's buffer is
        # summed into itself, so it is also the result).
        self.flat = [torch.zeros(nflat, **kw) for _ in range(self.S)]
        self.grads = _grad_views(self.flat[0], P, D)
        self.stream_of = [k % self.S for k in range(len(self.views))]
        # Capacity of each view's (Gaussian, tile) list from a probe forward;
        # one workspace per stream, sized for its largest view.
        caps = []
        for v in self.views:
            probe = Rasterizer(P, D, v.cam.width, v.cam.height, max_dups=64 * P + 4096, forward_only=True,
                               device=self.device)
            probe.forward(scene, v.cam, deform, v.t)
            caps.append(int(probe.stats()["num_dups"] * capacity_margin) + 4096)
            del probe
        torch.cuda.empty_cache()
        size = [0] * self.S
        for k, (v, cap) in enumerate(zip(self.views, caps)):
            need = max(Rasterizer.workspace_bytes(P, D, v.cam.width, v.cam.height, tile=s, max_dups=cap)
                       for s in TILE_SHAPES)
            size[self.stream_of[k]] = max(size[self.stream_of[k]], need)
        self.workspaces = [torch.empty(n, dtype=torch.uint8, device=self.device) for n in size]
        self.bufs = []
        for v in self.views:
            H, W = v.cam.height, v.cam.width
            self.bufs.append(dict(out=(torch.empty(3, H, W, **kw), torch.empty(H, W, **kw), torch.empty(H, W, **kw),
                                       torch.empty(H * W, D, **kw)),
                                  g_rgb=torch.full((3, H, W), 1e-3, **kw), g_feat=torch.full((H * W, D), 1e-3, **kw)))
        self.losses = torch.zeros(len(self.views), 2, **kw)
        self.scratch = torch.empty(len(self.views), 2, 1024, **kw)
        # Device error bits of each view (a workspace header is cleared by
        # every forward), copied out after each view.
        self.errs = torch.zeros(len(self.views), dtype=torch.int32, device=self.device)
        # Tile shape per view (autotuned per resolution, else 16x16).
        self.rasts, first = [], set()
        grads0 = _grad_views(self.flat[0], P, D)
        for k, (v, cap) in enumerate(zip(self.views, caps)):
            s = self.stream_of[k]
            shape = (16, 16)
            if autotuner is not None:
                b = self.bufs[k]
                shape = autotuner.pick(scene, deform, v.cam, v.t, cap, self.workspaces[s], grads0, b["g_rgb"],
                                       b["g_feat"])
            self.rasts.append(Rasterizer(P, D, v.cam.width, v.cam.height, tile=shape, max_dups=cap,
                                         device=self.device, auto_grow=False, accumulate=s in first,
                                         workspace=self.workspaces[s]))
            first.add(s)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.S)]
        self.graph = None

    @property
    def tile_shapes(self):
        return [r.tile for r in self.rasts]

    def _run_view(self, k: int, grads: dict):
        v, r, b = self.views[k], self.rasts[k], self.bufs[k]
        HW = v.cam.width * v.cam.height
        r.forward(self.scene, v.cam, self.deform, v.t, out=b["out"])
        _lib.fe_l1_loss_grad(b["out"][0], v.tgt_rgb, HW, b["g_rgb"], self.losses[k, 0:1], self.scratch[k, 0])
        _lib.fe_l1_loss_grad(b["out"][3], v.tgt_feat, HW, b["g_feat"], self.losses[k, 1:2], self.scratch[k, 1])
        r.backward(self.scene, v.cam, self.deform, v.t, b["g_rgb"], None, None, b["g_feat"], grads=grads)
        self.errs[k:k + 1].copy_(r.workspace[:4].view(torch.int32))

    def run(self):
        """All views: forward, L1 losses (RGB and features), backward; the
        gradients are summed into self.grads."""
        P, D = self.scene.P, self.scene.D
        if self.S == 1:
            for k in range(len(self.views)):
                self._run_view(k, self.grads)
            return
        main = torch.cuda.current_stream(self.device)
        start = torch.cuda.Event()
        start.record(main)
        done = []
        for s, st in enumerate(self.streams):
            st.wait_event(start)
            with torch.cuda.stream(st):
                g = _grad_views(self.flat[s], P, D)
                for k in range(len(self.views)):
                    if self.stream_of[k] == s:
                        self._run_view(k, g)
                e = torch.cuda.Event()
                e.record(st)
                done.append(e)
        for e in done:
            main.wait_event(e)
        _lib.fe_sum_f32(self.flat[0], self.flat, stream=main)

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
