"""Multi-rank host logic of the benchmark on CPU (two gloo ranks, no GPU): the envs shard
disjointly across ranks, the timed region's time is the slowest rank's, and the whole-job
throughput counts every rank's envs over that time."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = 2.0 + rank  # rank 1 is the slower one
        t = bench.max_over_ranks(seconds, world, "cpu")
        out[rank] = (t, bench.job_throughput(world, 4, 10, t), bench.shard_env_ids(rank, 4))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_envs_and_time_by_the_slowest_rank():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 3.0  # both ranks see the slowest rank's time
    assert res[0][1] == res[1][1] == 2 * 4 * 10 / 3.0
    ids0, ids1 = res[0][2], res[1][2]
    assert len(set(ids0) | set(ids1)) == 8 and not set(ids0) & set(ids1)
    assert bench.max_over_ranks(1.5, 1, "cpu") == 1.5
