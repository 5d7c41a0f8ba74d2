"""Multi-rank host logic of the benchmark on CPU (two gloo ranks, no GPU): the envs of an uneven
batch shard disjointly across ranks with balanced estimated cost, the timed region's time is the
slowest rank's, and the whole-job throughput counts every rank's env-steps over that time."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2503_05020_b300 import scenes as S


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = 2.0 + rank  # rank 1 is the slower one
        t = bench.max_over_ranks(seconds, world, "cpu")
        steps = bench.sum_over_ranks(40.0 + rank, world, "cpu")
        out[rank] = (t, bench.job_throughput(steps, t), bench.shard_env_ids(rank, world, 16, S.uneven_batch_cost))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_envs_and_time_by_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 3.0  # both ranks see the slowest rank's time
    assert res[0][1] == res[1][1] == 81.0 / 3.0  # every rank's env-steps over that time
    ids0, ids1 = res[0][2], res[1][2]
    assert set(ids0) | set(ids1) == set(range(32)) and not set(ids0) & set(ids1)
    c = [S.uneven_batch_cost(i) for i in range(32)]
    load = [sum(c[i] for i in ids) for ids in (ids0, ids1)]
    assert abs(load[0] - load[1]) <= max(c)  # greedy LPT: within one item of each other
    naive = [sum(c[:16]), sum(c[16:])]  # contiguous halves, for comparison
    assert abs(load[0] - load[1]) < abs(naive[0] - naive[1])
    assert bench.max_over_ranks(1.5, 1, "cpu") == 1.5


def test_lpt_shards_balance_an_uneven_batch():
    c = [S.uneven_batch_cost(i) for i in range(256)]
    t = sorted(c, reverse=True)
    for world in (2, 4, 8):
        bins = S.lpt_shards(c, world)
        assert sorted(i for b in bins for i in b) == list(range(256))
        load = [sum(c[i] for i in b) for b in bins]
        # LPT bound (Graham 1969): the largest load is at most 4/3 - 1/(3m) of the optimum, and the
        # optimum is at least the mean load and at least the largest item
        opt_lb = max(sum(c) / world, t[0])
        assert max(load) <= (4 / 3 - 1 / (3 * world)) * opt_lb + 1e-9
