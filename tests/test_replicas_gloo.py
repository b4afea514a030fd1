"""Multi-rank host logic of replica runs, on CPU with two gloo ranks.

Each rank samples independent chains from its own seed and the job time is the
slowest rank's; nothing else crosses ranks.  The checks: ranks get distinct seeds
whose momentum streams differ, every rank sees the maximum time, and the job rate
counts every rank's work against that time.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

import oracle  # noqa: E402
from paper_2507_14652_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.5 + rank                   # rank 1 is the slow one
        slowest = replicas.reduce_max(seconds, dist)
        seeds = [None] * world
        dist.all_gather_object(seeds, replicas.replica_seed(rank))
        out.put((rank, slowest, seeds))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_the_slowest_time_and_keep_chains_apart():
    world = 2
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, slowest, seeds in res:
        assert slowest == 2.5, (rank, slowest)
        assert seeds == [replicas.replica_seed(0), replicas.replica_seed(1)]
    s0, s1 = res[0][2]
    assert s0 != s1
    # the ranks' first momenta (chain 0, trajectory 0) come from different Philox keys
    m0 = oracle.momenta(s0, 0, 0, 8)
    m1 = oracle.momenta(s1, 0, 0, 8)
    assert not np.allclose(m0, m1)
    # whole-job rate: both ranks' units over the slowest rank's time
    C, L, steps = 16, 50, 10
    assert replicas.job_rate(world, C * L * steps, res[0][1]) == pytest.approx(2 * C * L * steps / 2.5)


def test_single_process_reduces_to_identity():
    assert replicas.reduce_max(3.25) == 3.25
    assert replicas.job_rate(1, 800, 2.0) == 400.0
    with pytest.raises(ValueError):
        replicas.job_rate(1, 800, 0.0)
