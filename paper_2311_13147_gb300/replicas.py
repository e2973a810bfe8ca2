"""Host logic for runs on several GPUs of one node (one process per GPU).

The cyclic path has no exchange step: every problem (and every batch of
problems) is independent.  A multi-GPU run is therefore a set of replicas:

* ``rank_seed``       -- the seed of a rank's own workload (weak scaling: every
                         rank solves a full workload of its own);
* ``shard_problems``  -- a balanced split of one problem list over ranks
                         (longest-processing-time by m^2, the per-sweep work),
                         for callers that divide a fixed batch instead;
* ``max_over_ranks``  -- the timing reduction of the benchmark (the slowest
                         rank defines the time of a step).

No collective touches the data path; ``max_over_ranks`` runs after the timed
region.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s workload; rank 0 keeps the base seed."""
    return int(base_seed) + 1000003 * int(rank)


def shard_problems(sizes, world: int):
    """Split problem indices over `world` ranks, balancing sum(m^2).

    sizes: block size m of every problem.  Greedy longest-processing-time:
    problems in decreasing m^2 (ties by index) go to the least loaded rank
    (ties to the lower rank).  Returns one sorted index list per rank.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]) ** 2, i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += int(sizes[i]) ** 2
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """All-reduce MAX of a per-rank scalar (no-op without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
