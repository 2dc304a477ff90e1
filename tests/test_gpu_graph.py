"""The whole step through the C ABI (index, seed cleaning, finding, duplicate removal, fit) captured
in one CUDA graph and replayed gives bit for bit what the eager calls give: the entry points
allocate nothing, synchronise nothing and keep no state between calls beyond caller buffers."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("adaptive", [0, 4])
def test_graph_replay_equals_eager_calls(adaptive):
    """With adaptive capacity the finder is two passes whose second takes its seeds (and their
    number) from device memory written by the first: the graph needs no host synchronisation."""
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as kf
    wl = synth.workload("duplicates", n_events=2, tracks_lo=800, tracks_hi=800)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    n, nh, lmax = dev["seed_hits"].shape[1], b.n_hits, wl.lmax
    cuda = torch.device("cuda")
    idx = kf.HitIndex(g, b.n_events, nh, cuda)
    keep = torch.ones(n, dtype=torch.int32, device=cuda)
    tkeep = torch.ones(n, dtype=torch.int32, device=cuda)
    dws = torch.empty(kf.dedup_workspace_size(n, lmax, nh), dtype=torch.uint8, device=cuda)
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, lmax, seed_keep=keep, adaptive_capacity=adaptive)
    fout = dict(hits=torch.empty((lmax, n), dtype=torch.int32, device=cuda),
                nhits=torch.empty(n, dtype=torch.int32, device=cuda),
                chi2=torch.empty(n, dtype=torch.float32, device=cuda),
                state=torch.empty((6, n), dtype=torch.float32, device=cuda),
                cov=torch.empty((21, n), dtype=torch.float32, device=cuda),
                status=torch.empty(n, dtype=torch.int32, device=cuda))
    fit = dict(state=torch.empty((6, n), dtype=torch.float32, device=cuda),
               cov=torch.empty((21, n), dtype=torch.float32, device=cuda),
               chi2=torch.empty(n, dtype=torch.float32, device=cuda),
               ndof=torch.empty(n, dtype=torch.int32, device=cuda),
               status=torch.empty(n, dtype=torch.int32, device=cuda))
    ws = torch.empty(kf.find_workspace_size(n, prm), dtype=torch.uint8, device=cuda)
    s = torch.cuda.Stream()

    def step():
        kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"], index=idx, stream=s)
        kf.clean_seeds(g, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], keep=keep,
                       workspace=dws, stream=s)
        kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm, out=fout,
                       workspace=ws, stream=s)
        kf.remove_duplicates(fout["hits"], fout["nhits"], fout["chi2"], fout["state"], dev["seed_event"], nh,
                             keep=tkeep, workspace=dws, stream=s)
        kf.fit_tracks(g, dev["hits"], dev["hit_surface"], fout["hits"], out=fit, stream=s)

    fkeys = ("hits", "nhits", "chi2", "state", "cov", "status")  # find_tracks also files its workspace in the dict
    bufs = lambda: (idx.bin_off, idx.sorted_ids, keep, tkeep, *(fout[k] for k in fkeys), *fit.values())
    outs = lambda: [t.clone() for t in bufs()]
    with torch.cuda.stream(s):
        step()
    torch.cuda.synchronize()
    ref = outs()
    for t in bufs():
        t.fill_(7)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step()
    graph.replay()
    torch.cuda.synchronize()
    got = outs()
    assert 0 < int((ref[2] == 0).sum()) < n  # cleaning removed some seeds
    for a, c in zip(ref, got):
        assert torch.equal(a.view(torch.int32) if a.dtype == torch.float32 else a,
                           c.view(torch.int32) if c.dtype == torch.float32 else c)
