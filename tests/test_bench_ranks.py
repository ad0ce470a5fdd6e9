"""Host logic of bench.py's multi-GPU form (replicas, no collective in the data path):
the slowest rank's timed region and the whole-job throughput, on world-size-2 gloo
process groups over CPU tensors."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 25.0 * rank                 # rank 1 is the slower replica
        m = bench.max_over_ranks(local_ms, torch.device("cpu"))
        v = bench.replica_throughput(382936, 20, world, m)
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_replicas_report_the_slowest_rank_and_whole_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, m, v in got:
        assert m == 125.0
        assert v == pytest.approx(2 * 382936 * 20 / 0.125 / 1e6)


def test_single_process_is_its_own_maximum():
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5
    assert bench.replica_throughput(10, 2, 1, 1000.0) == pytest.approx(2e-5)
