"""The N > 1 path of the benchmark on CPU: two gloo ranks. Ranks solve different seeded problems
(weak scaling, no collective on the data path); the step time is the slowest rank's (a MAX
all-reduce); the whole-job time per problem counts every rank's problems."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = 10.0 + 5.0 * rank              # a rank's own step time
    ms = bench.max_over_ranks(local, world, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.rank_seed(rank))
    out[rank] = (ms, seeds)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, seeds = res[r]
        assert ms == 15.0                  # every rank sees the slowest rank's time
        assert len(set(seeds)) == world    # different problems on every rank


def test_single_rank_and_whole_job_time():
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    # 2 ranks x 3 steps x 2 problems in 120 ms: 10 ms a problem for the whole job
    assert bench.whole_job_ms_per_problem(120.0, 3, 2, 2) == 10.0
