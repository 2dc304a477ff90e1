"""Multi-rank host logic on CPU (gloo, world size 2): event sharding covers every event exactly
once with balanced load, weak scaling gives each rank its own events, and the reported step time is
the max over ranks. No GPU and no data-path collective are involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1906_02253_gb300 import shard


def test_shard_events_partition_and_balance():
    rng = np.random.default_rng(3)
    counts = rng.integers(2000, 20001, size=100)
    for world in (1, 2, 3, 4, 8):
        parts = [shard.shard_events(counts, world, r) for r in range(world)]
        allv = np.sort(np.concatenate(parts))
        assert np.array_equal(allv, np.arange(100))
        loads = [counts[p].sum() for p in parts]
        assert max(loads) - min(loads) <= counts.max()  # greedy LPT bound


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synth
        wl = synth.workload("find", n_events=1, tracks_lo=50, tracks_hi=50)
        seed = shard.rank_seed(wl.seed, rank)
        b = synth.generate(wl, seed=seed)
        step_ms = 10.0 + 5.0 * rank  # stand-in for a measured step time
        n_seeds = len(b.seeds()[1])
        results[rank] = (seed, float(b.hits[:, 0].sum()), shard.max_over_ranks(step_ms), n_seeds,
                         shard.sum_over_ranks(n_seeds))
    finally:
        dist.destroy_process_group()


def test_weak_scaling_ranks_and_max_time():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    results = manager.dict()
    mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
    r0, r1 = results[0], results[1]
    assert r0[0] != r1[0]            # different generator seeds: different events per rank
    assert r0[1] != r1[1]
    assert r0[2] == r1[2] == 15.0    # both ranks report the slowest rank's time
    assert r0[4] == r1[4] == r0[3] + r1[3]  # the job's seeds: every rank's own count
