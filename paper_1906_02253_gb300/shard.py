"""Host-side logic for running the path on several GPUs, one process per GPU.

Events are independent and seeds never share state (the paper processes seeds in parallel without
marking used hits, Sec. 3.2), so the work shards by events with no exchange on the data path. Two
modes: weak scaling (every rank reconstructs its own batch of events, generated with a rank-specific
seed) and strong scaling (a fixed batch split across ranks by greedy longest-processing-time on the
events' track counts). The only collective is the max over ranks of the measured step time.
"""
from __future__ import annotations

import numpy as np


def rank_seed(base_seed: int, rank: int) -> int:
    """Generator seed of rank `rank` under weak scaling (rank 0 keeps the workload's own seed)."""
    return int(base_seed) + 1000 * int(rank)


def shard_events(track_counts, world: int, rank: int):
    """Events of `rank` when a fixed batch is split over `world` ranks: events taken in decreasing
    track count, each given to the rank with the least work so far (ties: lowest rank). Returns the
    sorted event indices of this rank."""
    counts = np.asarray(track_counts, dtype=np.int64)
    load = np.zeros(world, dtype=np.int64)
    owner = np.empty(len(counts), dtype=np.int64)
    for e in np.argsort(-counts, kind="stable"):
        r = int(np.argmin(load))
        owner[e] = r
        load[r] += counts[e]
    return np.nonzero(owner == rank)[0]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank value (e.g. the step time) over the process group; the value itself when
    no group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    """Sum of a per-rank value (e.g. the seeds a rank processed) over the process group; the value
    itself when no group is initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
