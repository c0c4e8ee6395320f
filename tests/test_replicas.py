"""Multi-rank host logic of the replica runs, as two gloo ranks on the CPU.

The GPU runs launch one process per GPU; their only exchange is host-side
(barrier, max of the timed seconds, sum of the units).  Here two CPU processes
run that code with different per-rank numbers and check the whole-job rate,
the maxima and the sharding of a job list.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1901_02492_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    replicas.init("gloo")
    r, w, local = replicas.dist_info()
    replicas.barrier()
    secs = 1.0 + rank                          # rank 1 is the slower one
    units = 100.0 * (rank + 1)
    rate, total, slowest = replicas.whole_job_rate(units, secs)
    mx = replicas.max_over_ranks([rank, -rank, 0.5 * rank])
    share = list(replicas.shard(10, r, w))
    replicas.barrier()
    replicas.finish()
    out.put((rank, r, w, local, rate, total, slowest, mx, share))


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shares = []
    for rank, r, w, local, rate, total, slowest, mx, share in res:
        assert (r, w, local) == (rank, 2, rank)
        assert total == 300.0 and slowest == 2.0 and rate == pytest.approx(150.0)
        assert mx == [1.0, 0.0, 0.5]
        shares += share
    assert shares == list(range(10))


@pytest.mark.parametrize("n,world", [(0, 1), (10, 1), (10, 3), (64, 8), (5, 8), (2000, 7)])
def test_shard_covers_every_unit_once(n, world):
    got = [list(replicas.shard(n, r, world)) for r in range(world)]
    flat = [u for s in got for u in s]
    assert flat == list(range(n))
    sizes = [len(s) for s in got]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_is_identity():
    assert replicas.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert replicas.whole_job_rate(50.0, 2.0) == (25.0, 50.0, 2.0)
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)
