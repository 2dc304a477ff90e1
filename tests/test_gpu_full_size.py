"""Parity at the benchmark's full sizes, in the launch configuration the benchmark times.

The GPU finds tracks for every seed of the full workloads (100 events; 200 events with disks and
noise; 100 events with the material map; 20 events in the field map) with the
autotuned block size, candidate capacity and adaptive capacity (calibrated on the first quarter of
the events, as the benchmark does) and fits every simulated track; the FP64 oracle then computes a seeded random sample of 20,000
seeds and 20,000 tracks one by one, and the sample is held to the parity bars: hit lists identical
on >= 99.9% of seeds, efficiency within 0.1%, every track with an identical hit list
carrying the same fitted state (1e-4) and chi2 (1e-3), fitted tracks within the fit bars.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from bench import calibration_events
from test_gpu_parity import _assert_track_state_parity

pytestmark = pytest.mark.gpu

FLOOR = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])
N_SAMPLE = 20000


def _rel(p_gpu, p_ora):
    d = p_gpu.astype(np.float64) - p_ora
    d[:, 4] = (d[:, 4] + np.pi) % (2 * np.pi) - np.pi
    return np.abs(d) / np.maximum(np.abs(p_ora), FLOOR)


@pytest.mark.parametrize("wl_name", ["fit_batched", "hi_occ", "material", "field"])
def test_full_size_parity_on_sampled_seeds_and_tracks(wl_name):
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as kf
    wl = synth.workload(wl_name)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
    n_cal = int(np.searchsorted(dev["seed_event"].cpu().numpy(), calibration_events(b.n_events)))
    cal_s = dev["seed_hits"][:, :n_cal].contiguous()
    cal_e = dev["seed_event"][:n_cal].contiguous()
    prm, _ = kf.autotune_find(g, idx, dev["hits"], dev["hit_surface"], cal_s, cal_e, prm)
    out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    fit_block, _ = kf.autotune_fit(g, dev["hits"], dev["hit_surface"], dev["track_hits"])
    fit = kf.fit_tracks(g, dev["hits"], dev["hit_surface"], dev["track_hits"], block_threads=fit_block)
    torch.cuda.synchronize()
    n = dev["seed_hits"].shape[1]
    assert n > 100_000

    rng = np.random.default_rng(1906)
    s = np.sort(rng.choice(n, N_SAMPLE, replace=False))
    sh, st = b.seeds()
    og = oracle.Geometry(wl)
    r = oracle.find(og, b, sh[s], b.track_event[st][s])
    gh = out["hits"].cpu().numpy().T[s]
    same = (gh == r["hits"]).all(axis=1)
    assert same.mean() >= 0.999, same.mean()
    g_status = out["status"].cpu().numpy()[s]
    assert np.array_equal(g_status, r["status"])
    e_g = oracle.efficiency(b, st[s], gh, out["nhits"].cpu().numpy()[s])[0]
    e_o = oracle.efficiency(b, st[s], r["hits"], r["n_hits"])[0]
    assert abs(e_g - e_o) <= 0.001
    ok = same & (r["status"] == 0)
    _assert_track_state_parity(out["state"].cpu().numpy().T[s][ok], out["chi2"].cpu().numpy()[s][ok],
                               r["p"][ok], r["cov"][ok], r["chi2"][ok])

    t = np.sort(rng.choice(b.n_tracks, N_SAMPLE, replace=False))
    f = oracle.fit(og, b.hits, b.hit_surface, b.track_hits[t])
    assert np.array_equal(fit["status"].cpu().numpy()[t], f["status"])
    assert np.array_equal(fit["ndof"].cpu().numpy()[t], f["ndof"])
    okf = f["status"] == 0
    relf = _rel(fit["state"].cpu().numpy().T[t][okf], f["p"][okf])
    assert relf.max() < 1e-4, relf.max(axis=0)
    fc2 = fit["chi2"].cpu().numpy()[t][okf]
    assert (np.abs(fc2 - f["chi2"][okf]) / np.maximum(f["chi2"][okf], 1.0)).max() < 1e-3


def test_full_size_seed_cleaning_and_duplicate_removal_chain():
    """The overlap workload at full size (219 k combinatorial seeds): the GPU's cleaning flags
    equal the oracle's on >= 99.9% of all seeds, and the whole chain (cleaning, finding, removal)
    gives the oracle's efficiency and duplicate rate within 0.1%."""
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as kf
    wl = synth.workload("duplicates")
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    keep = kf.clean_seeds(g, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"])
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, seed_keep=keep)
    out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    kd = kf.remove_duplicates(out["hits"], out["nhits"], out["chi2"], out["state"], dev["seed_event"], b.n_hits)
    torch.cuda.synchronize()
    sh, st = b.seeds()
    ev = b.track_event[st]
    og = oracle.Geometry(wl)
    ok = oracle.clean_seeds(sh, ev, oracle.seed_params(og, b, sh))
    gk = keep.cpu().numpy()
    assert len(sh) > 200_000 and (gk == ok).mean() >= 0.999
    k = np.nonzero(ok)[0]
    r = oracle.find(og, b, sh[k], ev[k])
    okd = np.zeros_like(ok)
    okd[k] = oracle.remove_duplicates(r["hits"], r["n_hits"], r["chi2"], r["p"][:, 4], r["p"][:, 5], ev[k])
    o_hits = np.full((len(sh), wl.lmax), -1, np.int32)
    o_hits[k] = r["hits"]
    o_nh = np.zeros(len(sh), np.int32)
    o_nh[k] = r["n_hits"]
    g_hits = out["hits"].cpu().numpy().T
    g_nh = out["nhits"].cpu().numpy()
    gkd = gk * kd.cpu().numpy()
    e_g, d_g = oracle.track_rates(b, st, np.ones(len(st), bool), gkd, track_sim=oracle.majority_sim(b, g_hits, g_nh))
    e_o, d_o = oracle.track_rates(b, st, np.ones(len(st), bool), okd, track_sim=oracle.majority_sim(b, o_hits, o_nh))
    assert abs(e_g - e_o) <= 0.001 and abs(d_g - d_o) <= 0.001


@pytest.mark.parametrize("wl_name,net,top_n,margin,window", [("learned", "mlp_learned.npz", 1, 0.0, False),
                                                             ("learned", "mlp_learned.npz", 4, 0.0, False),
                                                             ("hi_occ", "mlp_hi_occ.npz", 2, 0.0, False),
                                                             ("hi_occ", "mlp_hi_occ.npz", 4, 0.0, False),
                                                             ("hi_occ", "mlp_hi_occ.npz", 2, 0.7, False),
                                                             ("hi_occ", "mlp_hi_occ.npz", 2, 0.5, True)])
def test_full_size_learned_finding_on_sampled_seeds(wl_name, net, top_n, margin, window):
    """The learned proposal at full size, in the autotuned launch configuration the benchmark's
    learned-versus-plain comparison uses: hit lists identical to the FP64 oracle's (same network,
    same top_n, score margin and window rule) on >= 99.9% of a 20,000-seed sample, efficiency within
    0.1%."""
    import os
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as kf
    wl = synth.workload(wl_name)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    z = np.load(os.path.join(os.path.dirname(kf.__file__), "data", net))
    buf = kf.mlp_buffer(z["weights"], z["mean"], z["sd"])
    lp = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, mlp=buf, top_n=top_n, score_margin=margin,
                        window_ranking=window)
    n_cal = int(np.searchsorted(dev["seed_event"].cpu().numpy(), calibration_events(b.n_events)))
    lp, _ = kf.autotune_find(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"][:, :n_cal].contiguous(),
                             dev["seed_event"][:n_cal].contiguous(), lp)
    out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], lp)
    torch.cuda.synchronize()
    n = dev["seed_hits"].shape[1]
    s = np.sort(np.random.default_rng(2253).choice(n, N_SAMPLE, replace=False))
    sh, st = b.seeds()
    w = (z["weights"].astype(np.float64), z["mean"].astype(np.float64), z["sd"].astype(np.float64))
    r = oracle.find(oracle.Geometry(wl), b, sh[s], b.track_event[st][s], mlp=w, top_n=top_n, score_margin=margin,
                    window=window)
    gh = out["hits"].cpu().numpy().T[s]
    same = (gh == r["hits"]).all(axis=1)
    assert same.mean() >= 0.999, same.mean()
    e_g = oracle.efficiency(b, st[s], gh, out["nhits"].cpu().numpy()[s])[0]
    e_o = oracle.efficiency(b, st[s], r["hits"], r["n_hits"])[0]
    assert abs(e_g - e_o) <= 0.001
