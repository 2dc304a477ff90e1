"""Pins of the oracle's seed cleaning (Sec. 3.2: duplicate seeds of one particle removed before
finding, from hit identity and the seed direction) and duplicate-track removal (Sec. 4: duplicate
tracks from several seeds per particle), CPU only.

The oracle decides through an inverted index hit -> items; the pins decide by brute force over
all pairs on small inputs, and by hand on constructed cases.
"""
import numpy as np

import oracle
import synth


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _brute_clean(seeds, event, params, dphi, dtheta):
    n = len(seeds)
    keep = np.ones(n, np.int32)
    for j in range(n):
        if np.isnan(params[j, 1]):
            continue
        hj = {h for h in seeds[j] if h >= 0}
        for i in range(j):
            if event[i] != event[j] or not hj & {h for h in seeds[i] if h >= 0}:
                continue
            if abs(_wrap(params[i, 1] - params[j, 1])) < dphi and abs(params[i, 2] - params[j, 2]) < dtheta:
                keep[j] = 0
                break
    return keep


def _brute_dedup(hits, nh, chi2, phi, theta, event, dphi, dtheta):
    n = len(hits)
    keep = np.ones(n, np.int32)
    for j in range(n):
        hj = [h for h in hits[j] if h >= 0]
        for i in range(n):
            if i == j or event[i] != event[j]:
                continue
            better = (nh[i], -chi2[i], -i) > (nh[j], -chi2[j], -j)
            shared = sum(1 for h in hj if h in set(hits[i]))
            if better and 2 * shared > len(hj) and abs(_wrap(phi[i] - phi[j])) < dphi \
                    and abs(theta[i] - theta[j]) < dtheta:
                keep[j] = 0
                break
    return keep


def test_seed_cleaning_equals_brute_force_on_random_seeds():
    rng = np.random.default_rng(11)
    n = 400
    seeds = rng.integers(0, 150, size=(n, 3)).astype(np.int32)
    seeds[rng.random((n, 3)) < 0.05] = -1
    event = rng.integers(0, 2, n).astype(np.int32)
    # directions clustered so that many hit-sharing pairs are near the cuts
    params = np.stack([rng.normal(0, 1, n), _wrap(rng.integers(0, 4, n) * 0.015 + rng.normal(0, 0.01, n) + 3.13),
                       1.0 + rng.integers(0, 3, n) * 0.04 + rng.normal(0, 0.02, n)], axis=1)
    params[rng.random(n) < 0.03] = np.nan
    keep = oracle.clean_seeds(seeds, event, params, 0.02, 0.05)
    want = _brute_clean(seeds, event, params, 0.02, 0.05)
    assert np.array_equal(keep, want)
    assert 0.1 < (keep == 0).mean() < 0.9  # both decisions occur


def test_seed_cleaning_constructed_cases():
    p = np.array([[0.5, 1.0, 1.2], [0.5, 1.0, 1.2], [0.5, 1.0 + np.pi, 1.2], [0.5, 1.01, 1.2],
                  [0.5, 1.01, 1.2], [0.5, 1.025, 1.2], [0.5, -np.pi + 0.005, 1.2], [0.5, np.pi - 0.005, 1.2]])
    seeds = np.array([[1, 2, 3], [1, 2, 3], [1, 4, 5], [9, 10, 3], [11, 12, 13], [9, 14, 15], [20, 21, 22],
                      [20, 23, 24]], np.int32)
    event = np.array([0, 0, 0, 0, 0, 0, 0, 0], np.int32)
    keep = oracle.clean_seeds(seeds, event, p, 0.02, 0.05)
    # 1: a copy of 0; 2: shares hit 1 but points the other way; 3: agrees with 0 through hit 3;
    # 4: shares nothing; 5: agrees with 3 (removed itself) through hit 9 but not with 0;
    # 7: agrees with 6 across phi = +-pi
    assert keep.tolist() == [1, 0, 1, 0, 1, 0, 1, 0]
    event2 = event.copy()
    event2[1] = 1  # the copy in another event is kept
    assert oracle.clean_seeds(seeds, event2, p, 0.02, 0.05)[1] == 1
    # a seed with no direction is neither removed nor a reason to remove
    p2 = p.copy()
    p2[0] = np.nan
    k2 = oracle.clean_seeds(seeds, event, p2, 0.02, 0.05)
    assert k2[0] == 1 and k2[1] == 1 and k2[3] == 0  # 3 is now removed by 1, through hit 3
    assert oracle.clean_seeds(seeds[:0], event[:0], p[:0]).shape == (0,)


def test_duplicate_removal_equals_brute_force_on_random_tracks():
    rng = np.random.default_rng(12)
    n, lmax = 250, 8
    base = rng.integers(0, 60, size=(40, lmax))
    src = rng.integers(0, 40, n)
    hits = base[src].copy()
    hits = np.where(rng.random((n, lmax)) < 0.3, rng.integers(60, 400, size=(n, lmax)), hits)
    for t in range(n):  # distinct hits within a track, -1 padded at the end
        u = list(dict.fromkeys(int(h) for h in hits[t] if h >= 0))[: rng.integers(3, lmax + 1)]
        hits[t] = u + [-1] * (lmax - len(u))
    hits = hits.astype(np.int32)
    nh = (hits >= 0).sum(axis=1).astype(np.int32)
    chi2 = rng.integers(0, 5, n).astype(np.float64)  # ties
    phi = _wrap(src * 0.3 + rng.normal(0, 0.012, n))
    theta = 1.0 + (src % 5) * 0.2 + rng.normal(0, 0.03, n)
    event = (src % 2).astype(np.int32)
    keep = oracle.remove_duplicates(hits, nh, chi2, phi, theta, event, 0.02, 0.05)
    want = _brute_dedup(hits, nh, chi2, phi, theta, event, 0.02, 0.05)
    assert np.array_equal(keep, want)
    assert 0.1 < (keep == 0).mean() < 0.9


def test_duplicate_removal_constructed_cases():
    h = np.array([[1, 2, 3, 4, -1, -1], [1, 2, 3, 9, -1, -1], [1, 2, 7, 8, -1, -1], [1, 2, 3, 4, 5, 6],
                  [30, 31, 32, -1, -1, -1], [30, 31, 33, -1, -1, -1]], np.int32)
    nh = (h >= 0).sum(axis=1).astype(np.int32)
    chi2 = np.array([1.0, 2.0, 0.5, 9.0, 3.0, 3.0])
    phi = np.zeros(6)
    theta = np.ones(6)
    ev = np.zeros(6, np.int32)
    keep = oracle.remove_duplicates(h, nh, chi2, phi, theta, ev, 0.02, 0.05)
    # 3 has the most hits; 0 and 1 share 4 and 3 of their 4 hits with it; 2 shares exactly half
    # (not more) with 3 and with 0; 4 and 5 tie on hits and chi2: the lower index wins
    assert keep.tolist() == [0, 0, 1, 1, 1, 0]
    phi2 = phi.copy()
    phi2[3] = 0.5  # the long track points elsewhere: 0 is best of the rest
    assert oracle.remove_duplicates(h, nh, chi2, phi2, theta, ev, 0.02, 0.05).tolist() == [1, 0, 1, 1, 1, 0]


def test_track_rates_counts_per_simulated_track():
    class B:
        n_tracks = 4
        track_nhits = np.array([12, 12, 5, 12])
    st = np.array([0, 0, 1, 2, 2, 3])
    matched = np.array([1, 1, 0, 1, 1, 0], bool)
    assert oracle.track_rates(B, st, matched) == (1 / 3, 1 / 3)  # ref: 0, 1, 3 (2 is short)
    assert oracle.track_rates(B, st, matched, keep=[1, 0, 1, 1, 1, 1]) == (1 / 3, 0.0)


def test_majority_matching_follows_the_hits():
    class B:
        track_nhits = np.array([12, 12, 12])
        hit_sim = np.array([0, 0, 0, 1, 1, 1, 1, -1, 2, 2])
    h = np.array([[0, 1, 2, 3, -1], [3, 4, 5, 0, 1], [3, 4, 7, 0, 1], [8, 9, 7, -1, -1], [7, -1, -1, -1, -1]])
    nh = (h >= 0).sum(axis=1)
    # 0: 3 of 4 from sim 0; 1: 3 of 5 from sim 1; 2: 2 of 5 at most; 3: 2 of 3 from sim 2; 4: noise
    assert oracle.majority_sim(B, h, nh, min_hits=3).tolist() == [0, 1, -1, 2, -1]
    assert oracle.majority_sim(B, h, nh, min_hits=4).tolist() == [0, 1, -1, -1, -1]


def test_cleaning_and_dedup_on_overlap_workload():
    """Combinatorial seeds from module overlaps: most seeds are duplicates. Cleaning removes them at
    a small efficiency cost; without cleaning the duplicate track rate is large, and the
    duplicate-track removal takes it down without losing tracks (tracks matched to the sim track
    holding most of their hits)."""
    wl = synth.workload("duplicates", n_events=1, tracks_lo=600, tracks_hi=600)
    b = synth.generate(wl)
    sh, st = b.seeds()
    g = oracle.Geometry(wl)
    ev = b.track_event[st]
    assert len(sh) > 1.8 * len(np.unique(st))
    keep = oracle.clean_seeds(sh, ev, oracle.seed_params(g, b, sh))
    r = oracle.find(g, b, sh, ev)
    ms = oracle.majority_sim(b, r["hits"], r["n_hits"])
    eff_all, dup_all = oracle.track_rates(b, st, ms >= 0, track_sim=ms)
    eff_cl, dup_cl = oracle.track_rates(b, st, ms >= 0, keep, track_sim=ms)
    assert dup_all > 0.4 and dup_cl < 0.01
    assert eff_all - eff_cl < 0.005
    kd = oracle.remove_duplicates(r["hits"], r["n_hits"], r["chi2"], r["p"][:, 4], r["p"][:, 5], ev)
    eff_dd, dup_dd = oracle.track_rates(b, st, ms >= 0, kd, track_sim=ms)
    assert dup_dd < 0.05 * dup_all and eff_all - eff_dd < 0.002
    # the whole chain: duplicate removal over the tracks of the cleaned seeds
    k = np.nonzero(keep)[0]
    kd2 = oracle.remove_duplicates(r["hits"][k], r["n_hits"][k], r["chi2"][k], r["p"][k, 4], r["p"][k, 5], ev[k])
    chain = np.zeros_like(keep)
    chain[k] = kd2
    eff_ch, dup_ch = oracle.track_rates(b, st, ms >= 0, chain, track_sim=ms)
    assert dup_ch <= dup_cl and eff_cl - eff_ch < 0.002
