"""The data-parallel exchange step of view-sharded training, on CPU ranks
(gloo): each rank takes a contiguous shard of the views, sums its views'
parameter gradients in view order, and the exchange sums the ranks' sums.
The per-view gradients are the FP64 oracle's reverse pass of small scenes,
rounded to float32 (what a rank's renderer hands over).

* ``ordered``: every rank ends with the same bits as one process adding the
  ranks' partial sums in rank order.
* ``allreduce``: the backend's sum, within 1e-6 relative of that, and the
  same on every rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2503_06161_gb300 import dist as pdist  # noqa: E402
from paper_2503_06161_gb300 import synth  # noqa: E402

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh", "feat")
NVIEWS = 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene():
    sc = synth.make_scene(40, 4, (-0.6, -0.5, 2.0), (0.6, 0.5, 3.0), seed=12)
    sc.log_scales[:] += np.float32(1.0)
    df = synth.make_deform(40, C=32, R=6, bbox_min=(-1, -1, 1.5), bbox_max=(1, 1, 3.5), full_heads=True,
                           head_std=0.05, seed=13)
    return sc, df


def _view_grads(v):
    """float32 gradients of view v (its own camera, time and upstream
    gradients) from the FP64 oracle."""
    from oracle import oracle as O
    sc, df = _scene()
    rng = np.random.default_rng(100 + v)
    cam = synth.make_camera(24, 20, 22.0, rotation=synth.random_rotation(rng, 0.1),
                            translation=[0.03 * v, -0.02, 0.05])
    pix = O.all_pixels(cam.width, cam.height)
    n = len(pix)
    g = O.backward(sc, cam, df, v / (NVIEWS - 1), (0, 0, 0), pix, rng.normal(size=(n, 3)), rng.normal(size=n) * 0.1,
                   rng.normal(size=n), rng.normal(size=(n, sc.D)))
    return {k: torch.tensor(g[k], dtype=torch.float32).contiguous() for k in KEYS}


def _rank(rank, world, port, out_dir, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = pdist.shard(NVIEWS, world, rank)
        acc = None
        for v in range(lo, hi):
            g = _view_grads(v)
            acc = g if acc is None else {k: acc[k] + g[k] for k in KEYS}
        ex = pdist.GradExchange(world, mode=mode)
        tensors = [acc[k] for k in KEYS]
        ex.exchange(tensors)
        torch.save({k: t for k, t in zip(KEYS, tensors)}, os.path.join(out_dir, f"{mode}_r{rank}.pt"))
    finally:
        dist.destroy_process_group()


def _reference(world):
    """One process: each shard's views summed in view order, then the shards
    in rank order, all in float32."""
    per_view = [_view_grads(v) for v in range(NVIEWS)]
    parts = []
    for r in range(world):
        lo, hi = pdist.shard(NVIEWS, world, r)
        acc = per_view[lo]
        for v in range(lo + 1, hi):
            acc = {k: acc[k] + per_view[v][k] for k in KEYS}
        parts.append(acc)
    ref = parts[0]
    for p in parts[1:]:
        ref = {k: ref[k] + p[k] for k in KEYS}
    return ref


@pytest.mark.parametrize("world", [2, 3])
def test_view_sharded_exchange_matches_single_process_sum(tmp_path, world):
    port = _free_port()
    for mode in ("ordered", "allreduce"):
        mp.start_processes(_rank, args=(world, port, str(tmp_path), mode), nprocs=world, join=True,
                           start_method="spawn")
        port += 1
    ref = _reference(world)
    assert all(float(ref[k].abs().max()) > 0 for k in KEYS)
    for r in range(world):
        got = torch.load(tmp_path / f"ordered_r{r}.pt")
        for k in KEYS:
            assert torch.equal(got[k], ref[k]), (r, k)
        ar = torch.load(tmp_path / f"allreduce_r{r}.pt")
        ar0 = torch.load(tmp_path / "allreduce_r0.pt")
        for k in KEYS:
            assert torch.equal(ar[k], ar0[k]), (r, k)        # every rank the same
            den = torch.clamp(ref[k].abs(), min=float(ref[k].pow(2).mean().sqrt()) + 1e-30)
            assert float(((ar[k] - ref[k]).abs() / den).max()) <= 1e-6, k


def test_shards_cover_every_view_once():
    for n in (0, 1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            got = [pdist.shard(n, world, r) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))             # contiguous
            sizes = [hi - lo for lo, hi in got]
            assert max(sizes) - min(sizes) <= 1                                 # balanced
    with pytest.raises(ValueError):
        pdist.shard(4, 2, 2)


def test_single_rank_exchange_is_the_identity():
    t = torch.arange(6, dtype=torch.float32)
    pdist.GradExchange(1).exchange([t])
    assert torch.equal(t, torch.arange(6, dtype=torch.float32))


def test_ordered_sum_on_cpu_is_left_to_right():
    rng = np.random.default_rng(0)
    bufs = [torch.tensor(rng.normal(size=1000).astype(np.float32)) for _ in range(11)]
    out = torch.empty(1000)
    pdist.ordered_sum(bufs, out)
    ref = bufs[0].clone()
    for b in bufs[1:]:
        ref = ref + b
    assert torch.equal(out, ref)
