"""bench.py --gpus N runs N independent replicas of the workload (one cavity
per rank, no collective on the data path); the job's time is the slowest
rank's and its rate counts every rank's steps.  Two gloo ranks on the CPU
exercise that host-side logic."""
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


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank measured a different time; all of them see the slowest
        ms = bench.max_over_ranks(100.0 + 25.0 * rank, world, device="cpu")
        out[rank] = (ms, bench.replica_seed(rank), bench.whole_job_rate(3, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_count_all_steps():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 125.0
    assert out[0][1] != out[1][1]  # replicas simulate different seeded cavities
    assert out[0][2] == out[1][2] == pytest.approx(3 * 2 / 0.125)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_rate(10, 1, 500.0) == pytest.approx(20.0)
