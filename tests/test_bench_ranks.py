"""The multi-rank path of bench.py (one independent system per rank, weak
scaling), on CPU: two gloo ranks with different local times agree on the
slowest rank's time and on a job throughput that counts both ranks' work."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 100.0 * (rank + 1)            # rank 1 is the slow one
        ms, value = bench.job_throughput(ms_local, 4, 2.0e12, world, torch.device("cpu"))
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_both():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    slow_ms = 200.0 / 4                          # the slowest rank, per step
    for rank in range(world):
        ms, value = res[rank]
        assert ms == pytest.approx(slow_ms)
        assert value == pytest.approx(2.0e12 * world / (slow_ms * 1e-3) / 1e12)


def test_one_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    ms, value = bench.job_throughput(120.0, 3, 1.0e12, 1)
    assert ms == pytest.approx(40.0)
    assert value == pytest.approx(1.0e12 / 0.040 / 1e12)
