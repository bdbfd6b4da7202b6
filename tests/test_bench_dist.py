"""The bench's multi-rank host logic on CPU: two gloo ranks.

bench.py shards independent problems across ranks (weak scaling, no
data-path collective) and reduces only its timings, taking the maximum over
ranks; these tests run that logic in two processes without a GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench.rank_info()
        p = bench.rank_problem(r)
        local_ms = 100.0 + 37.0 * r                     # rank 1 is the slow one
        t = bench.max_over_ranks(local_ms, w)
        value = bench.whole_job_rate(p.n * p.steps, w, t / 1e3)
        out[rank] = (r, w, lr, p.n, p.steps, float(p.u0[:64].sum()), t, value)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_problems_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, w, lr, n, steps, head, t, value) in res.items():
        assert (r, w, lr) == (rank, world, rank)
        assert t == 137.0                                # max over ranks, on every rank
        assert value == pytest.approx(n * steps * world / 0.137)
    # same shape, different seeded data on each rank (independent problems)
    assert res[0][3:5] == res[1][3:5]
    assert res[0][5] != res[1][5]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(5.0, 1) == 5.0
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0
    assert np.array_equal(bench.rank_problem(0).u0, bench.rank_problem(0).u0)
