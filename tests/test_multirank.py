"""The N>1 host path of bench.py on CPU: two gloo ranks (processes) run the
replica logic -- each rank's timestamp, the max-over-ranks step time, the
whole-job rate -- exactly as the GPU ranks do, and the reference arm runs on
rank 0 alone."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.replica_time(0.5, rank, world)
        ms = 2.0 + 3.0 * rank          # rank 1 is the slower one
        dist.barrier()
        worst = bench.max_over_ranks(ms, world, torch.device("cpu"))
        rate = bench.whole_job_rate(worst, world)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{t} {worst} {rate}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slowest_time_and_render_distinct_timestamps(tmp_path):
    world = 2
    mp.start_processes(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [tuple(float(x) for x in open(tmp_path / f"r{r}.txt").read().split()) for r in range(world)]
    ts = [r[0] for r in res]
    assert ts == [0.5, 0.0]                       # replicas spread over [0, 1)
    assert all(r[1] == 5.0 for r in res)          # every rank reports the slowest rank's time
    assert all(r[2] == pytest.approx(world * 1000.0 / 5.0) for r in res)   # units of all ranks / that time


def test_single_rank_is_the_identity():
    assert bench.replica_time(0.3, 0, 1) == 0.3
    assert bench.max_over_ranks(1.25, 1, None) == 1.25
    assert bench.whole_job_rate(2.0, 1) == 500.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class A:
        workload, t, steps, warmup = bench.WORKLOAD, 0.5, 1, 0
    assert bench.run_reference(A(), 2, 1) is None   # rank 1 exits at once, without work or output
    assert capsys.readouterr().out == ""
