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
