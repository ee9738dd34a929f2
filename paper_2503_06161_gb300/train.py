"""One training iteration of FE-4DGS on the device (Sec. 3.3, Sec. 3.4, Sec. 4.1):
deformation query at time t, render forward (RGB, depth, D-channel
features), L1 RGB loss, decoder D -> 256 with the L1 feature loss (Eq. 10,
fused forward + reverse), the weighted depth and TV terms of Eq. 11, render
reverse, and an Adam step on every Gaussian parameter, the decoder and (with
the full FST module) the planes and every MLP weight, under the paper's
exponential learning-rate schedules.

Every step of the iteration runs in the library's kernels; this module only
owns the device buffers and sequences the C-ABI calls on the current stream,
with no host synchronisation inside a step.

    tr = Trainer.from_numpy(scene, camera, deform, decoder_w, decoder_b)
    tr.step(t, target_rgb, target_features)       # losses stay on the device
"""
from __future__ import annotations

import torch

from . import _lib, density
from .decoder import Decoder
from .fst import FSTDeform
from .optim import Adam, exp_lr
from .raster import DeformField, GaussianScene, Rasterizer, camera_struct

# Loss weights of Eq. 11 (RGB, depth, feature, TV).
LAMBDA_RGB, LAMBDA_DEPTH, LAMBDA_FEAT, LAMBDA_TV = 1.0, 0.01, 1.0, 0.03

# Initial per-group learning rates.  Position, grid and deformation follow
# the paper's hyperparameter table (SCARED column) and decay log-linearly to
# the final rates of SCHEDULE over SCHEDULE_STEPS (the table's position LR
# max steps); the other groups keep a constant rate.
LR = dict(means=1.6e-4, log_scales=5e-3, quats=1e-3, opacity_logits=5e-2, sh=2.5e-3, feat=2.5e-3,
          dec_weight=1e-3, dec_bias=1e-3, grid=1.6e-3, deformation=8e-5)
SCHEDULE = dict(means=1.6e-6, grid=1.6e-5, deformation=8e-7)
SCHEDULE_STEPS = 3000


class Trainer:
    def __init__(self, masters: dict, sh_degree: int, cam, deform: DeformField | None, decoder: Decoder,
                 bf16_storage: bool = True, max_dups: int | None = None, lr: dict | None = None, device="cuda",
                 fst: FSTDeform | None = None, schedule: bool = True, density_stats: bool = False,
                 grad_exchange=None):
        """masters: float32 device tensors means [P,3], log_scales [P,3],
        quats [P,4], opacity_logits [P], sh [P,16,3], feat [P,D].  deform:
        the single-level field evaluated inside the renderer, or fst: the
        full FST module (Sec. 3.2) run around it (not both).
        density_stats: gather the screen-space gradient statistics of
        adaptive density control every iteration (densify_and_prune).
        grad_exchange: a dist.GradExchange of data-parallel training; every
        step sums the ranks' gradients with it before the Adam update."""
        if deform is not None and fst is not None:
            raise ValueError("one deformation model: deform or fst")
        self.m = masters
        self.fst = fst
        self.schedule = bool(schedule)
        self.lr = dict(LR, **(lr or {}))
        P, D = masters["means"].shape[0], masters["feat"].shape[1]
        self.P, self.D = int(P), int(D)
        self.cam = cam if isinstance(cam, _lib.fe_camera) else camera_struct(cam)
        self.deform = deform
        self.dec = decoder
        self.bf16 = bf16_storage
        lr = dict(LR, **(lr or {}))
        # Storage the renderer reads: bf16 copies of SH and features,
        # refreshed by every Adam step.
        if bf16_storage:
            self.sh_store = masters["sh"].to(torch.bfloat16)
            self.feat_store = masters["feat"].to(torch.bfloat16)
        else:
            self.sh_store, self.feat_store = masters["sh"], masters["feat"]
        self.scene = GaussianScene(masters["means"], masters["log_scales"], masters["quats"],
                                   masters["opacity_logits"], self.sh_store, self.feat_store, sh_degree)
        W, H = self.cam.width, self.cam.height
        self.HW = W * H
        self.device = device
        self.rast = self._rasterizer(max_dups)
        kw = dict(dtype=torch.float32, device=device)
        self.out = (torch.empty(3, H, W, **kw), torch.empty(H, W, **kw), torch.empty(H, W, **kw),
                    torch.empty(self.HW, self.D, **kw))
        self.feat_bf = torch.empty(self.HW, self.D, dtype=torch.bfloat16, device=device)
        self.g_rgb = torch.empty(3, H, W, **kw)
        self.g_depth = torch.empty(H, W, **kw)
        # L_rgb, L_feat, lambda_depth * L_depth, lambda_TV * L_TV
        self.losses = torch.zeros(4, **kw)
        self.scratch = torch.empty(3, 1024, **kw)
        self.dec_out = (self.losses[1:2], torch.empty(self.HW, self.D, **kw), torch.empty(256, self.D, **kw),
                        torch.empty(256, **kw))
        self.grads = self._grad_buffers()
        self.dec_w32 = decoder.weight.float()
        groups = [dict(param=masters[k], lr=lr[k]) for k in ("means", "log_scales", "quats", "opacity_logits")]
        groups.append(dict(param=masters["sh"], lr=lr["sh"], param_bf16=self.sh_store if bf16_storage else None))
        groups.append(dict(param=masters["feat"], lr=lr["feat"],
                           param_bf16=self.feat_store if bf16_storage else None))
        groups.append(dict(param=self.dec_w32, lr=lr["dec_weight"], param_bf16=decoder.weight))
        groups.append(dict(param=decoder.bias, lr=lr["dec_bias"]))
        self.opt = Adam(groups)
        self.opt_fst = None
        if fst is not None:
            self.opt_fst = Adam([dict(param=fst.planes, lr=lr["grid"]), dict(param=fst.mlp, lr=lr["deformation"])])
        self.steps = 0
        self.exchange = grad_exchange
        self.dec.workspace(self.HW)
        self.stats = density.DensityStats(self.P, device) if density_stats else None

    def _rasterizer(self, max_dups: int | None) -> Rasterizer:
        """Rasterizer for the current P; without a capacity, one probe
        forward at t = 0.5 sizes the duplicate list (1.5x plus slack)."""
        W, H = self.cam.width, self.cam.height
        if max_dups is None:
            probe = Rasterizer(self.P, self.D, W, H, device=self.device, max_dups=64 * self.P + 4096,
                               forward_only=True)
            probe.forward(self.fst.forward(self.scene, 0.5) if self.fst is not None else self.scene, self.cam,
                          self.deform, 0.5)
            max_dups = int(probe.stats()["num_dups"] * 1.5) + 4096
            del probe
        return Rasterizer(self.P, self.D, W, H, max_dups=max_dups, device=self.device, auto_grow=False)

    def _grad_buffers(self) -> dict:
        P, D = self.P, self.D
        kw = dict(dtype=torch.float32, device=self.device)
        return dict(means=torch.empty(P, 3, **kw), log_scales=torch.empty(P, 3, **kw),
                    quats=torch.empty(P, 4, **kw), opacity_logits=torch.empty(P, **kw),
                    sh=torch.empty(P, 16, 3, **kw), feat=torch.empty(P, D, **kw))

    GAUSS_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh", "feat")

    def densify_and_prune(self, extent: float, normals: torch.Tensor | None = None,
                          grad_thresh: float = density.GRAD_THRESH, min_opacity: float = density.MIN_OPACITY,
                          generator: torch.Generator | None = None, max_dups: int | None = None) -> int:
        """Adaptive density control from the statistics gathered since the
        last call: clone / split / prune every parameter, the bf16 render
        copies and the Adam moments (new Gaussians start with zero moments),
        then rebuild every buffer sized by P.  dense_scale = percent dense
        (0.01) x extent.  normals: [P,2,3] N(0,1) draws placing split
        children (drawn with `generator` when not given).  Returns the new P;
        reads it back (one host sync)."""
        if self.stats is None:
            raise RuntimeError("construct the Trainer with density_stats=True")
        P = self.P
        if normals is None:
            normals = torch.randn(P, 2, 3, generator=generator, device=self.device, dtype=torch.float32)
        params = {k: self.m[k] for k in self.GAUSS_KEYS}
        if self.bf16:
            params["sh_store"], params["feat_store"] = self.sh_store, self.feat_store
        state = {}
        for i, k in enumerate(self.GAUSS_KEYS):
            state[k + ".m"], state[k + ".v"] = self.opt.groups[i]["m"], self.opt.groups[i]["v"]
        new_p, new_s, n = density.densify(params, state, self.stats, normals, grad_thresh,
                                          density.PERCENT_DENSE * float(extent), min_opacity)
        for k in self.GAUSS_KEYS:
            self.m[k] = new_p[k]
        if self.bf16:
            self.sh_store, self.feat_store = new_p["sh_store"], new_p["feat_store"]
        else:
            self.sh_store, self.feat_store = self.m["sh"], self.m["feat"]
        for i, k in enumerate(self.GAUSS_KEYS):
            g = self.opt.groups[i]
            g["param"], g["m"], g["v"] = self.m[k], new_s[k + ".m"], new_s[k + ".v"]
        self.opt.groups[4]["param_bf16"] = self.sh_store if self.bf16 else None
        self.opt.groups[5]["param_bf16"] = self.feat_store if self.bf16 else None
        self.P = n
        self.scene = GaussianScene(self.m["means"], self.m["log_scales"], self.m["quats"], self.m["opacity_logits"],
                                   self.sh_store, self.feat_store, self.scene.sh_degree)
        if self.fst is not None:
            self.fst.resize(n)
        self.grads = self._grad_buffers()
        self.rast = None
        self.rast = self._rasterizer(max_dups)
        self.stats.reset(n)
        return n

    def trained_grads(self) -> list:
        """The gradient tensors of every trained parameter (the data-parallel
        exchange sums these over the ranks)."""
        out = [self.grads[k] for k in self.GAUSS_KEYS] + [self.dec_out[2], self.dec_out[3]]
        if self.fst is not None:
            out += [self.fst.d_planes, self.fst.d_mlp]
        return out

    def reset_opacity(self, max_opacity: float = density.RESET_OPACITY):
        """Cap every opacity at max_opacity and restart its Adam moments."""
        density.reset_opacity(self.m["opacity_logits"], max_opacity)
        self.opt.groups[3]["m"].zero_()
        self.opt.groups[3]["v"].zero_()

    @classmethod
    def from_numpy(cls, sc, cam, df=None, dec_w=None, dec_b=None, device="cuda", bf16_storage=True, **kw):
        f = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
        masters = dict(means=f(sc.means), log_scales=f(sc.log_scales), quats=f(sc.quats),
                       opacity_logits=f(sc.opacity_logits), sh=f(sc.sh).reshape(sc.P, 16, 3), feat=f(sc.feat))
        deform = DeformField.from_numpy(df, device) if df is not None else None
        dec = Decoder(torch.as_tensor(dec_w).to(torch.bfloat16).to(device), f(dec_b))
        return cls(masters, int(sc.sh_degree), cam, deform, dec, bf16_storage=bf16_storage, device=device, **kw)

    def forward_backward(self, t: float, tgt_rgb: torch.Tensor, tgt_dec: torch.Tensor,
                         tgt_depth: torch.Tensor | None = None, events=None):
        """Losses and gradients of one view at time t (no parameter update):
        L1 RGB, the decoder's L1 feature loss, and (with a depth target) the
        weighted L1 depth loss of Eq. 11.  events: optional CUDA events
        recorded after the deformation, the losses, the render reverse and
        the FST reverse (profiling)."""
        rec = (lambda i: events[i].record()) if events is not None else (lambda i: None)
        scene = self.fst.forward(self.scene, t) if self.fst is not None else self.scene
        rec(0)
        self.rast.forward(scene, self.cam, self.deform, t, out=self.out, feat_bf16=self.feat_bf)
        _lib.fe_l1_loss_grad(self.out[0], tgt_rgb, self.HW, self.g_rgb, self.losses[0:1], self.scratch[0])
        self.dec.l1(self.feat_bf, tgt_dec, out=self.dec_out)
        g_depth = None
        if tgt_depth is not None:
            # lambda_depth * mean |depth - target|: the L1 kernel's row count
            # HW / lambda_depth gives the weighted loss and gradient.
            _lib.fe_l1_loss_grad(self.out[1], tgt_depth, round(self.HW / LAMBDA_DEPTH), self.g_depth,
                                 self.losses[2:3], self.scratch[1])
            g_depth = self.g_depth
        rec(1)
        self.rast.backward(scene, self.cam, self.deform, t, self.g_rgb, g_depth, None, self.dec_out[1],
                           grads=self.grads)
        if self.stats is not None:
            self.stats.record(self.rast)
        rec(2)
        if self.fst is not None:
            # Deformed-Gaussian gradients -> canonical, planes and weights;
            # then lambda_TV * L_TV on the planes.
            self.fst.backward(self.scene, t, self.grads)
            self.fst.tv(LAMBDA_TV, self.losses[3:4], self.scratch[2])
        rec(3)

    def step(self, t: float, tgt_rgb: torch.Tensor, tgt_dec: torch.Tensor,
             tgt_depth: torch.Tensor | None = None, events=None) -> torch.Tensor:
        """One training iteration; returns the device tensor
        [L_rgb, L_feat, lambda_depth * L_depth, lambda_TV * L_TV] (depth 0
        without a depth target, TV 0 without the FST module)."""
        self.forward_backward(t, tgt_rgb, tgt_dec, tgt_depth, events)
        g = self.grads
        if self.exchange is not None:
            self.exchange.exchange(self.trained_grads())
        lrs = None
        if self.schedule:
            lr = dict(self.lr, means=exp_lr(self.steps, self.lr["means"], SCHEDULE["means"], SCHEDULE_STEPS))
            lrs = [lr[k] for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "feat", "dec_weight",
                                   "dec_bias")]
        self.opt.step([g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], g["feat"],
                       self.dec_out[2], self.dec_out[3]], lrs)
        if self.fst is not None:
            fl = None
            if self.schedule:
                fl = [exp_lr(self.steps, self.lr[k], SCHEDULE[k], SCHEDULE_STEPS) for k in ("grid", "deformation")]
            self.opt_fst.step([self.fst.d_planes, self.fst.d_mlp], fl)
        self.steps += 1
        return self.losses
