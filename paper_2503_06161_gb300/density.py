"""Adaptive density control on the device: screen-space gradient statistics,
clone / split / prune, and the opacity reset (the procedure of the 3D
Gaussian splatting lineage; the paper's appendix hyperparameter table gives
its percent-dense fraction, 0.01 of the scene extent, and the opacity-reset
and prune intervals).

Every step runs in the library's kernels; this module allocates the output
buffers and reads back the new Gaussian count (one host sync per densify
call).

    stats = DensityStats(P)
    ...  rast.backward(...); stats.record(rast)          # every iteration
    params, state, n = densify(params, state, stats, normals, 2e-4, 0.01 * extent, 0.005)
"""
from __future__ import annotations

import torch

from . import _lib

PERCENT_DENSE = 0.01          # dense_scale = PERCENT_DENSE * scene extent (appendix table)
GRAD_THRESH = 2e-4            # mean NDC centre-gradient norm that triggers densification
MIN_OPACITY = 0.005           # prune below this opacity
RESET_OPACITY = 0.01          # opacity cap of the reset


class DensityStats:
    """Per-Gaussian sum of |dL/d(NDC centre)| over views and the view count."""

    def __init__(self, P: int, device="cuda"):
        self.accum = torch.zeros(int(P), dtype=torch.float32, device=device)
        self.count = torch.zeros(int(P), dtype=torch.int32, device=device)

    @property
    def P(self) -> int:
        return int(self.accum.shape[0])

    def record(self, rast, stream=None):
        """Add the view whose fe_render_backward ran last on rast's workspace."""
        if rast.P != self.P:
            raise ValueError("statistics and rasterizer disagree on P")
        _lib.fe_screen_grad_stats(rast.workspace, rast.P, rast.D, rast.width, rast.height, rast.opts, self.accum,
                                  self.count, stream)

    def reset(self, P: int | None = None):
        if P is not None and int(P) != self.P:
            dev = self.accum.device
            self.accum = torch.zeros(int(P), dtype=torch.float32, device=dev)
            self.count = torch.zeros(int(P), dtype=torch.int32, device=dev)
        else:
            self.accum.zero_()
            self.count.zero_()


def densify(params: dict, state: dict, stats: DensityStats, normals: torch.Tensor, grad_thresh: float,
            dense_scale: float, min_opacity: float, stream=None):
    """params: means [P,3], log_scales [P,3], quats [P,4], opacity_logits [P]
    (float32) and any other per-Gaussian tensors (float32 or bf16), each
    contiguous with P rows; state: per-Gaussian optimiser tensors (kept for
    survivors, zero for new Gaussians); normals [P,2,3] float32, the N(0,1)
    draws that place split children.  Returns (new params, new state, new P);
    the new tensors are the leading rows of buffers of 2P rows."""
    P = stats.P
    for k in ("means", "log_scales", "quats", "opacity_logits"):
        if k not in params:
            raise ValueError(f"params needs {k}")
    tensors = list(params.items()) + list(state.items())
    for k, v in tensors:
        if v.shape[0] != P or not v.is_contiguous():
            raise ValueError(f"{k}: expected a contiguous tensor with {P} rows")
    if normals.shape != (P, 2, 3) or normals.dtype != torch.float32:
        raise ValueError("normals must be float32 [P, 2, 3]")
    role = dict(means=_lib.FE_ATTR_MEANS, log_scales=_lib.FE_ATTR_LOG_SCALES)
    dev = params["means"].device
    st = _as_stream(stream, dev)
    # The inputs were produced on the caller's current stream: the densify
    # stream waits for it, and every buffer of this call is allocated and
    # zeroed on the densify stream itself, so the zero fill of the count is
    # ordered before the scan that writes it and no buffer returns to a pool
    # while the scatter may still use it.
    st.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(st):
        out_p = {k: torch.empty((2 * P,) + tuple(v.shape[1:]), dtype=v.dtype, device=v.device)
                 for k, v in params.items()}
        out_s = {k: torch.empty((2 * P,) + tuple(v.shape[1:]), dtype=v.dtype, device=v.device)
                 for k, v in state.items()}
        attrs = [(v, out_p[k], role.get(k, _lib.FE_ATTR_COPY)) for k, v in params.items()]
        attrs += [(v, out_s[k], _lib.FE_ATTR_STATE) for k, v in state.items()]
        new_P = torch.zeros(1, dtype=torch.int64, device=dev)
        ws = torch.empty(_lib.fe_densify_workspace_size(P), dtype=torch.uint8, device=dev)
        nrm = normals.contiguous()
        # One call moves at most 32 streams; more streams take further calls,
        # each repeating the (deterministic) decision and scan.
        for i in range(0, len(attrs), 32):
            chunk = attrs[i:i + 32]
            _lib.fe_densify(P, params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                            stats.accum, stats.count, nrm, grad_thresh, dense_scale, min_opacity, chunk, 2 * P,
                            new_P, ws, st)
    st.synchronize()  # the count was written on the densify stream
    cur = torch.cuda.current_stream(dev)
    if st != cur:
        # The outputs belong to the densify stream's pool; the caller goes on
        # using them on its current stream.
        for v in list(out_p.values()) + list(out_s.values()):
            v.record_stream(cur)
    n = int(new_P.item())
    return ({k: v[:n] for k, v in out_p.items()}, {k: v[:n] for k, v in out_s.items()}, n)


def _as_stream(stream, device):
    """torch stream object for None (the current stream), a torch stream, or
    a raw cudaStream_t handle (int)."""
    if stream is None:
        return torch.cuda.current_stream(device)
    if isinstance(stream, torch.cuda.Stream):
        return stream
    return torch.cuda.ExternalStream(int(stream), device=device)


def reset_opacity(logits: torch.Tensor, max_opacity: float = RESET_OPACITY, stream=None):
    """logits <- min(logits, logit(max_opacity)), in place."""
    _lib.fe_reset_opacity(logits, max_opacity, stream)
