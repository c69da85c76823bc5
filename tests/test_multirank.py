"""The benchmark's N > 1 path on CPU: two gloo ranks combine their times
the way bench.py does under torchrun (slowest rank, whole-job units)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    total_ms, value = bench.job_throughput(1000.0, my_ms, world, dist, "cpu")
    out.put((rank, total_ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_bench():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total_ms, value in res:
        assert total_ms == 150.0                      # the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 0.150)  # both ranks' units


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_throughput(10.0, 20.0, 1) == (20.0, 500.0)
