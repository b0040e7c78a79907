"""The multi-rank logic of bench.py on CPU: two gloo ranks (one process
each, rendezvous on 127.0.0.1) time different amounts of work; both get the
slowest rank's time, and the whole-job rate counts every rank's replica.
The reference arm does its work on rank 0 only."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        e2e_s = bench.max_over_ranks(2.0 - rank, dist, "cpu")
        dist.barrier()
        q.put((rank, bench.dist_env(), ms, bench.job_rate(world, 1000, 10, ms * 1e-3), e2e_s))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, env, ms, rate, e2e_s in out:
        assert env == (2, rank, rank)
        assert ms == 15.0 and e2e_s == 2.0
        # 2 replicas x 1000 nodes x 10 steps in the slowest rank's 15 ms
        assert rate == pytest.approx(2 * 1000 * 10 / 0.015 / 1e6)


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1, 1048576, 10, 1.0) == pytest.approx(10.48576)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    # a non-zero rank returns before building or running the oracle
    assert bench.run_reference(None) is None


def test_all_cores_oracle_replicas_aggregate():
    """The all-cores CPU baseline: one single-threaded oracle replica per
    core in its own spawned process; the aggregate counts every replica."""
    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as orc

    orc.build()
    rate, procs, steps, seconds = bench.oracle_rate_all_cores("delaunay_droplet_256x256", 0.3, 65536, procs=2)
    assert procs == 2 and steps >= 2 and seconds >= 0.3
    assert 0.0 < rate < 65536 * steps / 0.3 / 1e6
    assert bench.host_cores() >= 1
