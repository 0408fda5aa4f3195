"""The N>1 path of bench.py on CPU ranks (gloo, world size 2).

The transform shards by fields: every rank runs its own replica of the
workload with no data-path collective.  What crosses ranks is the barrier
around the timed region and the max-over-ranks of its duration, from which
the whole-job throughput (units of all ranks / slowest rank's time) follows.
Those helpers are exercised here on two gloo processes.
"""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert bench.dist_env() == (world, rank, rank)
    bench.barrier(world)
    t = bench.reduce_max(10.0 + 5.0 * rank, world)  # per-rank timed-region ms
    v = bench.job_throughput(fields_per_rank=548, steps=3, world=world, max_ms=t)
    bench.barrier(world)
    dist.destroy_process_group()
    out.put((rank, t, v))


def test_two_gloo_ranks_reduce_and_throughput():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks see the slowest rank's time, and the job throughput counts
    # the fields of both ranks over it
    assert [r[1] for r in res] == [15.0, 15.0]
    assert res[0][2] == res[1][2] == pytest.approx(2 * 548 * 3 / 0.015)


def test_single_rank_helpers_are_identity():
    import bench

    assert bench.reduce_max(3.5, 1) == 3.5
    bench.barrier(1)
    assert bench.job_throughput(fields_per_rank=4, steps=2, world=1, max_ms=1000.0) == pytest.approx(8.0)
