"""Torch-facing API of the semantic decoder (Sec. 3.3; feature loss Eq. 10).

The decoder is a 1x1 convolution from the D rendered feature channels to
256, run by the library's tensor-core kernel on BF16 operands with FP32
accumulation.  ``Decoder.l1`` fuses it with the L1 feature loss of Eq. 10
and the loss's reverse pass; the 256-channel map is never materialised.

    dec = Decoder.random(D=32, device="cuda")
    loss, d_feat, d_w, d_b = dec.l1(feat_bf16, target)          # scale 1/HW
"""
from __future__ import annotations

import torch

from . import _lib

COUT = 256


class Decoder:
    """Weights [256, D] bf16 and bias [256] float32 on the device."""

    def __init__(self, weight: torch.Tensor, bias: torch.Tensor):
        if weight.dtype != torch.bfloat16 or weight.dim() != 2 or weight.shape[0] != COUT:
            raise ValueError("weight must be a [256, D] bf16 tensor")
        if bias.dtype != torch.float32 or bias.shape != (COUT,):
            raise ValueError("bias must be a [256] float32 tensor")
        self.weight = weight.contiguous()
        self.bias = bias.contiguous()
        self._ws = None

    @property
    def D(self) -> int:
        return int(self.weight.shape[1])

    @classmethod
    def random(cls, D: int, device="cuda", seed: int = 0, w_std: float = 0.05, b_std: float = 0.0) -> "Decoder":
        g = torch.Generator().manual_seed(seed)
        w = (torch.randn(COUT, D, generator=g) * w_std).to(torch.bfloat16)
        b = torch.randn(COUT, generator=g) * b_std
        return cls(w.to(device), b.to(device))

    def workspace(self, HW: int) -> torch.Tensor:
        n = _lib.fe_decoder_workspace_size(HW, self.D)
        if n == 0:
            raise _lib.FeError("fe_decoder_workspace_size", 4)  # FE_ERR_UNSUPPORTED
        if self._ws is None or self._ws.numel() < n or self._ws.device != self.weight.device:
            self._ws = torch.empty(n, dtype=torch.uint8, device=self.weight.device)
        return self._ws

    def _args(self, feat: torch.Tensor) -> _lib.fe_decoder_args:
        if feat.dtype != torch.bfloat16 or feat.dim() != 2 or feat.shape[1] != self.D or not feat.is_contiguous():
            raise ValueError("feat must be a contiguous [HW, D] bf16 tensor")
        return _lib.make_decoder_args(feat, self.weight, self.bias)

    def forward(self, feat: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """out [HW, 256] float32 = feat W^T + b."""
        a = self._args(feat)
        if out is None:
            out = torch.empty(feat.shape[0], COUT, dtype=torch.float32, device=feat.device)
        _lib.fe_decode_forward(a, out, self.workspace(feat.shape[0]))
        return out

    def l1(self, feat: torch.Tensor, target: torch.Tensor, scale: float | None = None, out=None):
        """(loss [1], d_feat [HW, D], d_weight [256, D], d_bias [256]), all
        float32, for loss = scale * sum |decoder(feat) - target| (default
        scale 1/HW: Eq. 10).  target [HW, 256] bf16 or float32."""
        HW = feat.shape[0]
        if target.shape != (HW, COUT) or target.dtype not in (torch.bfloat16, torch.float32):
            raise ValueError("target must be [HW, 256] bf16 or float32")
        a = self._args(feat)
        dev = feat.device
        if out is None:
            out = (torch.empty(1, dtype=torch.float32, device=dev),
                   torch.empty(HW, self.D, dtype=torch.float32, device=dev),
                   torch.empty(COUT, self.D, dtype=torch.float32, device=dev),
                   torch.empty(COUT, dtype=torch.float32, device=dev))
        loss, d_feat, d_w, d_b = out
        s = (1.0 / HW if HW else 0.0) if scale is None else float(scale)
        _lib.fe_decode_l1(a, target.contiguous(), s, loss, d_feat, d_w, d_b, self.workspace(HW))
        return loss, d_feat, d_w, d_b

    def errors(self) -> int:
        return 0 if self._ws is None else _lib.fe_decoder_read_errors(self._ws)
