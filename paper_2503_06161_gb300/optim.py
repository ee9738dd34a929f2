"""Adam over the Gaussian parameters through the library's fused update
kernel (FP32 masters; optional bf16 copies for the renderer's storage).

    opt = Adam([dict(param=means, lr=1.6e-4), dict(param=sh32, lr=2.5e-3, param_bf16=sh_bf16), ...])
    opt.step([g_means, g_sh, ...])
"""
from __future__ import annotations

import torch

from . import _lib


class Adam:
    """Moments live on the device next to the parameters; the step count is
    a host integer (bias correction), so each call is one launch."""

    def __init__(self, groups, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
        if not 1 <= len(groups) <= 8:
            raise ValueError("1..8 parameter groups")
        self.groups = []
        for g in groups:
            p = g["param"]
            if p.dtype != torch.float32 or not p.is_contiguous():
                raise ValueError("parameters must be contiguous float32 masters")
            pb = g.get("param_bf16")
            if pb is not None and (pb.dtype != torch.bfloat16 or pb.numel() != p.numel()):
                raise ValueError("param_bf16 must be a bf16 tensor of the same size")
            self.groups.append(dict(param=p, lr=float(g["lr"]), param_bf16=pb, m=torch.zeros_like(p),
                                    v=torch.zeros_like(p)))
        self.beta1, self.beta2, self.eps = beta1, beta2, eps
        self.t = 0

    def step(self, grads, lrs=None):
        """One update; lrs (optional, one float per group) overrides the
        groups' learning rates for this and later steps (schedules)."""
        if len(grads) != len(self.groups):
            raise ValueError("one gradient per group")
        if lrs is not None:
            if len(lrs) != len(self.groups):
                raise ValueError("one learning rate per group")
            for g, lr in zip(self.groups, lrs):
                g["lr"] = float(lr)
        self.t += 1
        _lib.fe_adam_step([dict(g, grad=gr.contiguous()) for g, gr in zip(self.groups, grads)], self.t,
                          self.beta1, self.beta2, self.eps)


def exp_lr(step: int, lr_init: float, lr_final: float, max_steps: int) -> float:
    """Log-linear decay from lr_init to lr_final over max_steps (held at
    lr_final afterwards), the schedule form of the paper's hyperparameter
    table (initial / final rates, Appendix)."""
    import math
    r = min(max(step / max(max_steps, 1), 0.0), 1.0)
    return math.exp(math.log(lr_init) * (1.0 - r) + math.log(lr_final) * r)
