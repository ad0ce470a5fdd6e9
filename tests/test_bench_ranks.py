"""Host logic of bench.py's multi-GPU forms (no collective in the data path): replicas of
the headline workload, and the batched workload's problems split over the ranks; the
slowest rank's timed region, the summed leaves and the whole-job throughput, on
world-size-2 gloo process groups over CPU tensors."""
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


def _rank_shard(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ks = bench.shard_problems(64, rank, world)
        leaves = sum(1000 + k for k in ks)                # stand-in leaf counts per problem
        local_ms = 40.0 + 10.0 * rank
        total_ms = bench.max_over_ranks(local_ms, torch.device("cpu"))
        total = bench.sum_over_ranks(leaves, torch.device("cpu"))
        q.put((rank, ks, total, bench.sharded_throughput(total, 3, total_ms)))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_splits_every_problem_once_and_sums_the_leaves():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_shard, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    ks = sorted(k for _, kk, _, _ in got for k in kk)
    assert ks == list(range(64))
    total = sum(1000 + k for k in range(64))
    for rank, kk, t, v in got:
        assert t == total
        assert v == pytest.approx(total * 3 / 0.050 / 1e6)   # the slower rank's 50 ms


def test_shards_for_any_world_size():
    for world in (1, 2, 3, 4, 8):
        parts = [bench.shard_problems(64, r, world) for r in range(world)]
        assert sorted(k for p in parts for k in p) == list(range(64))
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
        if world > 1:
            # the batch alternates Dirichlet (even k) and cut-cell (odd k) problems: every
            # rank gets both kinds, in numbers that differ by at most one
            for p in parts:
                odd = sum(k % 2 for k in p)
                assert abs(odd - (len(p) - odd)) <= 1


def test_single_process_is_its_own_maximum():
    assert bench.max_over_ranks(7.5, torch.device("cpu")) == 7.5
    assert bench.replica_throughput(10, 2, 1, 1000.0) == pytest.approx(2e-5)
