"""The bench's multi-GPU path is replicas only: each rank runs the whole
evaluation and the job's value is (ranks x steps) over the slowest rank's
time.  Checked here with two gloo ranks on the CPU (no GPU involved): the
MAX over ranks and the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_seconds = [2.5, 4.0][rank]          # rank 1 is the slow replica
        slowest = bench.max_over_ranks(local_seconds, world, "cpu")
        out[rank] = (slowest, bench.whole_job_rate(5, world, slowest))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(2):
            slowest, rate = out[r]
            assert slowest == 4.0
            assert rate == pytest.approx(2 * 5 / 4.0)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.25, 1, "cpu") == 1.25
    assert bench.whole_job_rate(3, 1, 1.5) == pytest.approx(2.0)
