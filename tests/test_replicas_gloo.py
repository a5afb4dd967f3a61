"""Multi-process (N > 1) replica path of bench.py on the CPU: two gloo ranks
on 127.0.0.1, each with its own step time; every rank must see the slowest
rank's time, and the whole-job throughput counts every rank's pixels over
that time (weak scaling, no data-path collective)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank
    slowest = bench.max_over_ranks(dist, ms, "cpu")
    q.put((rank, slowest, bench.job_mpix_s(world, 2_073_600, slowest)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = sorted(q.get(timeout=5) for _ in range(world))
    for rank, slowest, mpix in res:
        assert slowest == pytest.approx(15.0)
        assert mpix == pytest.approx(2 * 2_073_600 / 0.015 / 1e6)
