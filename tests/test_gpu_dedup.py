"""Parity of the CUDA seed cleaning (Sec. 3.2) and duplicate-track removal (Sec. 4) with the oracle,
through the C ABI, and the finder's seed keep mask.

Cleaning compares seed directions the GPU computes in FP32 with the oracle's FP64 ones, so a pair
right at a cut may be decided differently: keep flags identical on >= 99.9% of seeds. Duplicate
removal on identical inputs (the oracle's tracks rounded to FP32 on both sides) is bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as k
    k.load_library()
    return k


@pytest.fixture(scope="module")
def overlap_events():
    wl = synth.workload("duplicates", n_events=2, tracks_lo=1500, tracks_hi=1500)
    b = synth.generate(wl)
    sh, st = b.seeds()
    return wl, b, sh, st


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t if dtype is None else t.to(dtype)).cuda()


def _gpu_dedup(kf, hits, nh, chi2, phi, theta, ev, n_hits, **kw):
    n, lmax = hits.shape
    state = np.zeros((6, n), np.float32)
    state[4], state[5] = phi, theta
    keep = kf.remove_duplicates(_dev(hits.T.astype(np.int32)), _dev(nh.astype(np.int32)), _dev(chi2.astype(np.float32)),
                                _dev(state), _dev(ev.astype(np.int32)), n_hits, **kw)
    return keep.cpu().numpy()


def test_clean_seeds_parity(kf, overlap_events):
    wl, b, sh, st = overlap_events
    dev = kf.to_device_event_batch(b)
    keep = kf.clean_seeds(kf.Geometry(wl), dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"])
    torch.cuda.synchronize()
    g = oracle.Geometry(wl)
    want = oracle.clean_seeds(sh, b.track_event[st], oracle.seed_params(g, b, sh))
    got = keep.cpu().numpy()
    assert (got == want).mean() >= 0.999, (got == want).mean()
    assert 0.4 < (want == 0).mean() < 0.7  # most combinatorial seeds are duplicates


def test_clean_seeds_other_cuts_and_edges(kf, overlap_events):
    wl, b, sh, st = overlap_events
    dev = kf.to_device_event_batch(b)
    geom = kf.Geometry(wl)
    g = oracle.Geometry(wl)
    pr = oracle.seed_params(g, b, sh)
    for dphi, dth in ((0.0, 0.05), (0.005, 0.01), (1e3, 1e3)):
        got = kf.clean_seeds(geom, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], dphi,
                             dth).cpu().numpy()
        want = oracle.clean_seeds(sh, b.track_event[st], pr, dphi, dth)
        assert (got == want).mean() >= 0.999
    empty = torch.empty((3, 0), dtype=torch.int32, device="cuda")
    assert kf.clean_seeds(geom, dev["hits"], dev["hit_surface"], empty, empty[0]).numel() == 0
    with pytest.raises(kf.KfError):
        kf.clean_seeds(geom, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], -1.0)


def test_remove_duplicates_bit_exact_on_oracle_tracks(kf, overlap_events):
    wl, b, sh, st = overlap_events
    ev = b.track_event[st]
    r = oracle.find(oracle.Geometry(wl), b, sh, ev)
    chi2 = r["chi2"].astype(np.float32)
    phi, theta = r["p"][:, 4].astype(np.float32), r["p"][:, 5].astype(np.float32)
    got = _gpu_dedup(kf, r["hits"], r["n_hits"], chi2, phi, theta, ev, len(b.hits))
    want = oracle.remove_duplicates(r["hits"], r["n_hits"], chi2.astype(np.float64), phi.astype(np.float64),
                                    theta.astype(np.float64), ev)
    assert np.array_equal(got, want)
    assert 0.4 < (want == 0).mean() < 0.7


def test_remove_duplicates_bit_exact_on_random_tracks_with_ties(kf):
    rng = np.random.default_rng(21)
    n, lmax = 3000, 12
    base = rng.integers(0, 800, size=(500, lmax))
    src = rng.integers(0, 500, n)
    hits = np.where(rng.random((n, lmax)) < 0.3, rng.integers(800, 6000, size=(n, lmax)), base[src])
    for t in range(n):
        u = list(dict.fromkeys(int(h) for h in hits[t]))[: rng.integers(3, lmax + 1)]
        hits[t] = u + [-1] * (lmax - len(u))
    hits = hits.astype(np.int32)
    nh = (hits >= 0).sum(axis=1).astype(np.int32)
    chi2 = rng.integers(0, 4, n).astype(np.float32)
    phi = ((src * 0.37 + rng.normal(0, 0.012, n) + np.pi) % (2 * np.pi) - np.pi).astype(np.float32)
    theta = (0.3 + (src % 7) * 0.35 + rng.normal(0, 0.03, n)).astype(np.float32)
    ev = (src % 3).astype(np.int32)
    got = _gpu_dedup(kf, hits, nh, chi2, phi, theta, ev, 6000)
    want = oracle.remove_duplicates(hits, nh, chi2.astype(np.float64), phi.astype(np.float64),
                                    theta.astype(np.float64), ev)
    assert np.array_equal(got, want)
    assert 0.1 < (want == 0).mean() < 0.9
    # no tracks, and an lmax above the compiled capacity
    assert _gpu_dedup(kf, hits[:0], nh[:0], chi2[:0], phi[:0], theta[:0], ev[:0], 6000).shape == (0,)
    with pytest.raises(kf.KfError):
        _gpu_dedup(kf, np.full((4, kf.KF_MAX_LMAX + 1), -1, np.int32), nh[:4], chi2[:4], phi[:4], theta[:4], ev[:4],
                   6000)


def test_find_with_seed_keep_mask(kf, overlap_events):
    """Removed seeds come out empty with status 2; kept seeds find what the oracle finds for them."""
    wl, b, sh, st = overlap_events
    ev = b.track_event[st]
    g = oracle.Geometry(wl)
    keep = oracle.clean_seeds(sh, ev, oracle.seed_params(g, b, sh))
    geom = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(geom, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, seed_keep=_dev(keep))
    out = kf.find_tracks(geom, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    rm = keep == 0
    assert np.all(gpu["status"][rm] == 2) and np.all(gpu["nhits"][rm] == 0) and np.all(gpu["hits"][:, rm] == -1)
    assert np.all(np.isnan(gpu["state"][:, rm]))
    k = np.nonzero(keep)[0]
    r = oracle.find(g, b, sh[k], ev[k])
    same = (gpu["hits"][:, k].T == r["hits"]).all(axis=1)
    assert same.mean() >= 0.999
    assert np.array_equal(gpu["status"][k], r["status"])


def test_clean_find_dedup_chain_rates_match_oracle(kf, overlap_events):
    """The whole chain on each side (GPU: its cleaning, finder and removal; oracle: its own), with
    efficiency and duplicate rate from the sim track holding most of each track's hits."""
    wl, b, sh, st = overlap_events
    ev = b.track_event[st]
    geom = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(geom, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    keep = kf.clean_seeds(geom, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"])
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, seed_keep=keep)
    out = kf.find_tracks(geom, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    kd = kf.remove_duplicates(out["hits"], out["nhits"], out["chi2"], out["state"], dev["seed_event"], len(b.hits))
    torch.cuda.synchronize()
    gk = (keep * kd).cpu().numpy()
    g_hits = out["hits"].cpu().numpy().T
    g_ms = oracle.majority_sim(b, g_hits, out["nhits"].cpu().numpy())
    g = oracle.Geometry(wl)
    ok = oracle.clean_seeds(sh, ev, oracle.seed_params(g, b, sh))
    k = np.nonzero(ok)[0]
    r = oracle.find(g, b, sh[k], ev[k])
    okd = np.zeros_like(ok)
    okd[k] = oracle.remove_duplicates(r["hits"], r["n_hits"], r["chi2"], r["p"][:, 4], r["p"][:, 5], ev[k])
    o_hits = np.full((len(sh), wl.lmax), -1, np.int32)
    o_hits[k] = r["hits"]
    o_nh = np.zeros(len(sh), np.int32)
    o_nh[k] = r["n_hits"]
    o_ms = oracle.majority_sim(b, o_hits, o_nh)
    assert (gk == okd).mean() >= 0.999
    e_g, d_g = oracle.track_rates(b, st, g_ms >= 0, gk, track_sim=g_ms)
    e_o, d_o = oracle.track_rates(b, st, o_ms >= 0, okd, track_sim=o_ms)
    assert abs(e_g - e_o) <= 0.001 and abs(d_g - d_o) <= 0.001
    assert e_o > 0.99 and d_o < 0.01
