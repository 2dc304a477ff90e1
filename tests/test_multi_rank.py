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


def _strong_worker(rank, world, port, results):
    """A rank of a fixed batch: its events by LPT on track counts, its sub-batch, the oracle's
    finding on it, hit ids mapped back to the whole batch."""
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import synth
        wl = synth.workload("find", n_events=5, tracks_lo=80, tracks_hi=400, seed=17)
        b = synth.generate(wl)
        counts = np.bincount(b.track_event, minlength=b.n_events)
        events = shard.shard_events(counts, world, rank)
        sub = b.select_events(events)
        sh, st = sub.seeds()
        f = oracle.find(oracle.Geometry(sub.wl), sub, sh, sub.track_event[st])
        # sub-batch hit ids back to the whole batch's
        so = b.slab_offsets.astype(np.int64)
        back = np.concatenate([np.arange(so[e * b.n_surf], so[(e + 1) * b.n_surf]) for e in events])
        hits = np.where(f["hits"] >= 0, back[np.maximum(f["hits"], 0)], -1)
        tracks = np.nonzero(np.isin(b.track_event, events))[0][st]
        n_seeds = len(st)
        results[rank] = (events.tolist(), tracks.tolist(), hits.tolist(), shard.sum_over_ranks(n_seeds))
    finally:
        dist.destroy_process_group()


def test_strong_scaling_shards_reproduce_single_rank_tracks():
    """Strong scaling: the two ranks' shares of one batch cover every event once, and the tracks
    each rank finds on its sub-batch are, hit for hit, the tracks found on the whole batch."""
    import oracle
    import synth
    world = 2
    port = _free_port()
    manager = mp.Manager()
    results = manager.dict()
    mp.spawn(_strong_worker, args=(world, port, results), nprocs=world, join=True)
    wl = synth.workload("find", n_events=5, tracks_lo=80, tracks_hi=400, seed=17)
    b = synth.generate(wl)
    sh, st = b.seeds()
    whole = oracle.find(oracle.Geometry(wl), b, sh, b.track_event[st])
    row = {int(t): i for i, t in enumerate(st)}
    events = sorted(results[0][0] + results[1][0])
    assert events == list(range(5))
    n = 0
    for r in range(world):
        ev, tracks, hits, total = results[r]
        assert total == len(st)
        for t, h in zip(tracks, hits):
            assert h == whole["hits"][row[t]].tolist(), (r, t)
            n += 1
    assert n == len(st)
