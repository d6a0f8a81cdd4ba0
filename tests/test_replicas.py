"""The N > 1 path of bench.py (replicas only: one chain does not shard) with
two gloo ranks on the CPU: every rank gets its own chain seeds, the job's
time is the slowest rank's, and the job's rate counts every rank's work."""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        t = bench.max_over_ranks(1.5 + r, w, device="cpu")
        seed = bench.replica_seed(42, r)
        seeds = bench.ensemble_replica_seeds([1000, 1001], r)
        every = [None] * w
        dist.all_gather_object(every, (seed, seeds))
        q.put((r, w, local, t, every, bench.job_rate(w, 100, t)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_on_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(2, _free_port(), q), nprocs=2, join=True, start_method="spawn")
    got = sorted(q.get() for _ in range(2))
    assert [g[0] for g in got] == [0, 1] and all(g[1] == 2 and g[2] == g[0] for g in got)
    for r, w, local, t, every, rate in got:
        assert t == pytest.approx(2.5)                       # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 100 / 2.5)          # both ranks' work over that time
        assert every == got[0][4]
    (s0, e0), (s1, e1) = got[0][4]
    assert (s0, s1) == (42, 43)                              # each replica its own chain
    assert set(e0).isdisjoint(e1)                            # and its own ensemble chains


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.job_rate(1, 50, 2.0) == 25.0
    assert bench.replica_seed(7, 0) == 7
