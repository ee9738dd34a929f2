"""Data-parallel training across GPUs: the views (timestamps, cameras) of a
training batch are split between the ranks of a process group, every rank
renders its own views forward and backward with its own replica of the
Gaussians and the deformation field, and ONE exchange step per iteration
sums the ranks' parameter gradients before the (identical) Adam step on
every rank.

The views are independent units (each is one rasterization pass, Sec. 3.3);
the paper trains on one GPU with one view per iteration (Sec. 4.1), so the
split is this library's own.  The exchanged gradients are those of every
trained tensor: the Gaussians (P x (3 + 3 + 4 + 1 + 48 + D) floats), the
decoder and, with the full FST module, its planes and weights.

Two exchanges:
  * ``ordered`` (default): an all-gather of the ranks' sums, then the sum
    taken in rank order on each rank -- every rank gets the same bits, the
    same as one process summing the ranks' partial sums in that order, on
    any backend (NCCL on GPUs, gloo on CPUs);
  * ``allreduce``: one sum all-reduce (the backend's reduction order).

    lo, hi = shard(V, world, rank)      # this rank's views
    ...  render views [lo, hi), gradients summed in view order into grads
    GradExchange(world).exchange(list_of_grad_tensors)
"""
from __future__ import annotations

import torch

from . import _lib


def shard(n: int, world: int, rank: int) -> tuple:
    """Contiguous share [lo, hi) of n items for `rank` of `world` ranks; the
    first n % world ranks take one item more."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need 0 <= rank < world and n >= 0")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def ordered_sum(bufs: list, out: torch.Tensor):
    """out = ((bufs[0] + bufs[1]) + bufs[2]) + ... in float32, elementwise;
    on the GPU in the library's fixed-order sum kernel, 8 sources a call."""
    if out.is_cuda:
        acc = bufs[0]
        i = 1
        while i < len(bufs):
            chunk = [acc] + bufs[i:i + 7]
            _lib.fe_sum_f32(out, chunk)
            acc = out
            i += 7
        if len(bufs) == 1:
            out.copy_(bufs[0])
        return out
    out.copy_(bufs[0])
    for b in bufs[1:]:
        out.add_(b)
    return out


class GradExchange:
    """The exchange step of view-parallel training for one process group."""

    def __init__(self, world: int | None = None, group=None, mode: str = "ordered"):
        import torch.distributed as dist
        if mode not in ("ordered", "allreduce"):
            raise ValueError("mode is 'ordered' or 'allreduce'")
        self.dist = dist
        self.group = group
        self.world = int(world) if world is not None else (dist.get_world_size(group) if dist.is_initialized() else 1)
        self.mode = mode
        self._scratch: dict = {}

    def exchange(self, tensors: list):
        """Replaces each float32 tensor (contiguous) by the sum over the ranks
        of its value on every rank; identity for one rank."""
        if self.world <= 1:
            return tensors
        for t in tensors:
            if t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError("gradients must be contiguous float32 tensors")
            flat = t.view(-1)
            if self.mode == "allreduce":
                self.dist.all_reduce(flat, op=self.dist.ReduceOp.SUM, group=self.group)
                continue
            key = (flat.numel(), flat.device)
            bufs = self._scratch.get(key)
            if bufs is None:
                bufs = [torch.empty_like(flat) for _ in range(self.world)]
                self._scratch[key] = bufs
            self.dist.all_gather(bufs, flat, group=self.group)
            ordered_sum(bufs, flat)
        return tensors
