"""The N-GPU benchmark runs independent replicas (no data-path collective):
its host logic -- a barrier, the max of the ranks' step times, the whole-job
throughput -- is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = bench.max_over_ranks(1.5 + rank, "cpu")          # rank 1 is the slower one
    out[rank] = (ms, bench.job_value(1_000_000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 2.5
        assert value == pytest.approx(2 * 1_000_000 / 2.5e-3 / 1e6)


def test_single_process_keeps_its_time():
    import bench
    assert bench.max_over_ranks(3.25, "cpu") == 3.25
    assert bench.job_value(5_000_000, 1, 1.0) == pytest.approx(5000.0)
