"""The multi-GPU path is replicas only: N independent runs, no data-path
collective.  What bench.py does across ranks (a barrier, the max of the
per-rank times, the whole-job rate) is checked here with two gloo ranks on
the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    job_ms = bench.max_over_ranks(local_ms, dist, device="cpu")
    rate = bench.job_rate(1.0e9, world, job_ms / 1000.0)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, job_ms, rate))


def test_two_replicas_take_the_slowest_time():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, job_ms, rate in res:
        assert job_ms == 150.0
        assert rate == pytest.approx(2 * 1.0e9 / 0.150)
    del torch


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.job_rate(3.0, 1, 1.5) == 2.0
