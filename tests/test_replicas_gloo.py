"""Host logic of the multi-GPU path (independent replicas, one process per
GPU): the whole-job rate is the work of all ranks over the slowest rank's
time, found by one all-reduce; the reference arm runs on rank 0 only.
Two CPU ranks under gloo; no GPU."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist, device="cpu")
        rate = bench.whole_job_rate(1000.0, world, slowest)
        out.put((rank, slowest, rate))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_slowest_rank_times_the_whole_job():
    ctx = mp.get_context("spawn")
    out = ctx.SimpleQueue()
    times = [0.5, 2.0]
    mp.start_processes(_rank, args=(2, _free_port(), times, out), nprocs=2, join=True, start_method="spawn")
    got = sorted(out.get() for _ in range(2))
    for rank, slowest, rate in got:
        assert slowest == 2.0
        assert rate == pytest.approx(2 * 1000.0 / 2.0)


def test_without_process_group_the_local_time_counts():
    import bench
    assert bench.max_over_ranks(1.25, None) == 1.25
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = bench.parse(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(args)
    assert buf.getvalue() == ""
