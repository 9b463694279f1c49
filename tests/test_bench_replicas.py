"""Multi-rank host logic of bench.py on CPU: two gloo ranks.

The path shards by cosmology ("replicas": no data-path collective), so what
runs across ranks is the job's bookkeeping: each rank's batch is a disjoint set
of seeded cosmologies, the job's time is the slowest rank's (all-reduce MAX),
and the job's throughput counts every rank's batches over that time.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    ids = bench.replica_request_ids(rank, 4)
    env = bench.env_rank()
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slowest, ids, env))


def test_two_gloo_ranks_share_the_slowest_time_and_disjoint_batches():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, ids0, env0), (r1, t1, ids1, env1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 15.0                       # max over ranks, seen by both
    assert set(ids0).isdisjoint(ids1) and len(ids0) == len(ids1) == 4
    assert env0 == (0, 0, 2) and env1 == (1, 1, 2)


def test_single_rank_and_throughput_bookkeeping():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5   # no process group needed at world 1
    assert bench.replica_request_ids(0, 3) == [1, 2, 3]
    assert bench.job_throughput(2, 256, 10, 0.5) == pytest.approx(10240.0)
