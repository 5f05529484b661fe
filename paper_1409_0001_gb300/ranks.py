"""Host-side helpers for running the coarse-graining path on several GPUs of one node.

The path has no exchange step between GPUs: independent snapshots (or independent
replicas of one workload) are assigned to ranks, each rank deposits and smooths its own
on its own GPU, and only scalars (the slowest rank's time, the units all ranks
processed) are combined.  One process per GPU, started by ``torch.distributed.run``;
the rank layout comes from the environment it sets.
"""
from __future__ import annotations

import os


def dist_env(environ=None):
    """(world_size, rank, local_rank) from the variables ``torch.distributed.run`` sets;
    (1, 0, 0) for a plain single-process run."""
    env = os.environ if environ is None else environ
    ws = int(env.get("WORLD_SIZE", "1"))
    rank = int(env.get("RANK", "0"))
    local = int(env.get("LOCAL_RANK", "0"))
    if ws < 1 or not 0 <= rank < ws or local < 0:
        raise ValueError("inconsistent rank layout: WORLD_SIZE=%d RANK=%d LOCAL_RANK=%d"
                         % (ws, rank, local))
    return ws, rank, local


def shard_by_cost(costs, world, rank):
    """Indices of the independent work items that ``rank`` of ``world`` owns.

    Longest-processing-time-first greedy: items in order of decreasing cost (ties by
    index) go one by one to the rank with the least assigned cost so far (ties to the
    lowest rank).  Deterministic, so every rank computes the same partition without
    communicating; the heaviest rank carries at most the mean load plus one item.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside world of %d" % (rank, world))
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += float(costs[i])
    return [i for i in range(len(costs)) if owner[i] == rank]


def reduce_scalar(x, op, device="cpu"):
    """``x`` combined over all ranks with ``op`` ("max" or "sum"), through a one-element
    all-reduce on ``device`` (the process group's backend decides which device works:
    "cuda" for NCCL, "cpu" for gloo).  Without an initialised process group it returns
    ``x`` unchanged."""
    import torch
    import torch.distributed as dist

    if op not in ("max", "sum"):
        raise ValueError("op must be 'max' or 'sum'")
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())
