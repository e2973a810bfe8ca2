"""Multi-process host logic on CPU (gloo, world size 2): replica seeds, sharding, timing reduction."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_13147_gb300 import replicas as R


def test_shard_problems_partitions_and_balances():
    sizes = [158, 8162, 4000, 4000, 300, 2048, 1, 7000, 3000, 3000, 512]
    for world in (1, 2, 3, 4):
        parts = R.shard_problems(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] ** 2 for i in p) for p in parts]
        # LPT bound: no rank exceeds the mean by more than the largest item
        assert max(loads) <= sum(loads) / world + max(s * s for s in sizes)
    assert R.shard_problems([5, 5], 4)[2:] == [[], []]
    with pytest.raises(ValueError):
        R.shard_problems([1], 0)


def test_rank_seed_distinct():
    seeds = {R.rank_seed(0, r) for r in range(8)}
    assert len(seeds) == 8 and R.rank_seed(7, 0) == 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [100 + 37 * i for i in range(23)]
        parts = R.shard_problems(sizes, world)
        mine = parts[rank]
        # every rank derives the same partition without communicating; check through a gather
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        ms = 10.0 + 5.0 * rank
        slowest = R.max_over_ranks(ms)
        out[rank] = (gathered, slowest, R.rank_seed(3, rank))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_run():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    g0, s0, seed0 = out[0]
    g1, s1, seed1 = out[1]
    assert g0 == g1
    assert sorted(g0[0] + g0[1]) == list(range(23)) and not set(g0[0]) & set(g0[1])
    assert s0 == s1 == 15.0
    assert seed0 != seed1


def test_max_over_ranks_without_group():
    assert R.max_over_ranks(3.5) == 3.5
