"""The multi-rank path on CPU: two gloo ranks shard a batch of jobs with no
data-path collective, and the whole-job throughput is the sum of the ranks'
work over the slowest rank's time (the benchmark's rule)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2311_01598_gb300 import dist as kd


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = list(range(13))
    mine = kd.shard(jobs, rank, world)
    seconds = 1.0 + rank          # rank 1 is the slower one
    rate = kd.job_throughput(len(mine), seconds)
    m = kd.max_over_ranks(seconds)
    dist.barrier()
    q.put((rank, mine, rate, m, kd.env_rank()))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_shard_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (r0, m0, rate0, mx0, env0), (r1, m1, rate1, mx1, env1) = out
    assert m0 + m1 == list(range(13)) and abs(len(m0) - len(m1)) <= 1
    assert rate0 == rate1 == pytest.approx(13 / 2.0)
    assert mx0 == mx1 == 2.0
    assert env0 == (0, 2, 0) and env1 == (1, 2, 1)


def test_shard_single_rank_and_uneven():
    assert kd.shard(list(range(5)), 0, 1) == list(range(5))
    parts = [kd.shard(list(range(10)), r, 4) for r in range(4)]
    assert sum(parts, []) == list(range(10)) and [len(p) for p in parts] == [3, 3, 2, 2]
    assert kd.max_over_ranks(3.5) == 3.5


def _tower_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nq, kp, N = 5, 3, 4
    parts = [kd.tower_partition(nq, kp, world, g) for g in range(world)]
    q0, q1, p0, p1 = parts[rank]
    # y: the rank's Q rows, each filled with its tower index
    y_own = torch.arange(q0, q1, dtype=torch.int64)[:, None].repeat(1, N)
    y_all = kd.all_gather_towers(y_own, [pt[1] - pt[0] for pt in parts])
    # w: [2][own special rows][N], tagged with polynomial and tower
    w_own = torch.stack([torch.arange(p0, p1, dtype=torch.int64)[:, None].repeat(1, N) + 100 * x for x in range(2)])
    w_all = kd.all_gather_towers(w_own, [pt[3] - pt[2] for pt in parts])
    q.put((rank, parts[rank], y_all.tolist(), w_all.tolist()))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_tower_partition_and_gathers():
    """Tower sharding's host side on two gloo ranks: the partition covers
    every Q and special tower once (uneven sizes), and both all-gathers
    assemble the rows in tower order on every rank."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_tower_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    (_, part0, y0, w0), (_, part1, y1, w1) = out
    assert part0 == (0, 3, 0, 2) and part1 == (3, 5, 2, 3)
    want_y = [[t] * 4 for t in range(5)]
    want_w = [[[t + 100 * x] * 4 for t in range(3)] for x in range(2)]
    assert y0 == y1 == want_y and w0 == w1 == want_w


def test_tower_partition_covers_every_tower():
    for nq, kp, world in ((24, 8, 4), (5, 3, 2), (7, 3, 4), (36, 12, 3)):
        parts = [kd.tower_partition(nq, kp, world, g) for g in range(world)]
        assert [t for q0, q1, _, _ in parts for t in range(q0, q1)] == list(range(nq))
        assert [t for _, _, p0, p1 in parts for t in range(p0, p1)] == list(range(kp))
        for nact in range(1, nq + 1):
            act = [kd.active_q(pt, nact) for pt in parts]
            assert [t for a, b in act for t in range(a, b)] == list(range(nact))
