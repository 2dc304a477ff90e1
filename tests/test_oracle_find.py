"""Pins of the oracle's combinatorial finder (CPU only).

The beam search is checked against plain search loops written here from the oracle's single-step
primitives (propagate, brute-force hit search, update): K = 1 is the greedy best-chi2 walk, and a
K larger than the number of branches is exhaustive enumeration. On clean sparse events every true
hit must be found. The binned and brute-force search modes give identical tracks.
"""
import numpy as np
import pytest

import oracle
import synth


def _seed_fit(g, b, ids):
    """Seed state at hit 1, then update with hit 1 and propagate + update through hits 2, 3."""
    p, C = oracle.seed(g, b.hits, b.hit_surface, ids)
    chi2 = 0.0
    for k, h in enumerate(ids):
        s = int(b.hit_surface[h])
        if k > 0:
            p, C, _, _ = oracle.propagate(g, p, C, s)
        p, C, c2 = oracle.update(g, p, C, s, b.hits[h])
        chi2 += c2
    return p, C, chi2


def _expand(g, b, wl, ev, p, C):
    """One step: next surface, prediction, and every passing hit (id, chi2), or None."""
    surf, _ = oracle.next_surface(g, p)
    if surf < 0:
        return None
    r = oracle.propagate(g, p, C, surf)
    if r is None:
        return None
    pp, CC = r[0], r[1]
    ids, c2 = oracle.search(g, b, pp, CC, ev, surf, wl.chi2_cut, brute=True)
    return surf, pp, CC, ids, c2


def _greedy(g, b, wl, seed_ids, ev, lmax):
    p, C, chi2 = _seed_fit(g, b, seed_ids)
    hits = list(seed_ids)
    n_miss = 0
    while len(hits) < lmax:
        e = _expand(g, b, wl, ev, p, C)
        if e is None:
            break
        surf, pp, CC, ids, c2 = e
        if len(ids):
            j = min(range(len(ids)), key=lambda i: (c2[i], ids[i]))
            p, C, _ = oracle.update(g, pp, CC, surf, b.hits[ids[j]])
            chi2 += c2[j]
            hits.append(int(ids[j]))
        elif n_miss < wl.max_miss:
            p, C = pp, CC
            n_miss += 1
            hits.append(-1)
        else:
            break
    return hits + [-1] * (lmax - len(hits))


def _enumerate(g, b, wl, seed_ids, ev, lmax):
    """Every branch of the search tree; best by (most hits, lowest chi2)."""
    p, C, chi2 = _seed_fit(g, b, seed_ids)
    leaves = []

    def rec(p, C, chi2, hits, n_miss, n_hits):
        if len(hits) >= lmax:
            leaves.append((-n_hits, chi2, hits))
            return
        e = _expand(g, b, wl, ev, p, C)
        if e is None:
            leaves.append((-n_hits, chi2, hits))
            return
        surf, pp, CC, ids, c2 = e
        if len(ids):
            for i in range(len(ids)):
                pn, Cn, _ = oracle.update(g, pp, CC, surf, b.hits[ids[i]])
                rec(pn, Cn, chi2 + c2[i], hits + [int(ids[i])], n_miss, n_hits + 1)
        elif n_miss < wl.max_miss:
            rec(pp, CC, chi2, hits + [-1], n_miss + 1, n_hits)
        else:
            leaves.append((-n_hits, chi2, hits))

    rec(p, C, chi2, list(seed_ids), 0, 3)
    leaves.sort(key=lambda x: (x[0], x[1]))
    best = leaves[0][2]
    return best + [-1] * (lmax - len(best)), len(leaves), leaves


def _tiny(wl_name, n_tracks, noise, seed):
    wl = synth.workload(wl_name, n_events=2, tracks_lo=n_tracks, tracks_hi=n_tracks, noise_frac=noise, seed=seed)
    return wl, oracle.Geometry(wl), synth.generate(wl)


@pytest.mark.parametrize("wl_name", ["find", "hi_occ"])
def test_k1_is_greedy_best_chi2(wl_name):
    wl, g, b = _tiny(wl_name, 25, 3.0, 21)
    sh, st = b.seeds()
    ev = b.track_event[st]
    f = oracle.find(g, b, sh, ev, k_max=1)
    for i in range(len(st)):
        ref = _greedy(g, b, wl, sh[i], ev[i], wl.lmax)
        assert f["hits"][i].tolist() == ref, i


def test_large_k_is_exhaustive_enumeration():
    """Dense noise (100 noise hits per signal hit) makes branches; with K above the number of
    leaves the beam search keeps everything and must return the enumeration's best."""
    wl, g, b = _tiny("find", 12, 100.0, 22)
    sh, st = b.seeds()
    ev = b.track_event[st]
    f = oracle.find(g, b, sh, ev, k_max=400)
    branched = 0
    for i in range(len(st)):
        best, n_leaves, _ = _enumerate(g, b, wl, sh[i], ev[i], wl.lmax)
        if n_leaves > 400:
            continue
        branched += n_leaves > 1
        assert f["hits"][i].tolist() == best, i
    assert branched >= 3


@pytest.mark.parametrize("wl_name", ["find", "hi_occ"])
def test_clean_sparse_events_find_every_true_hit(wl_name):
    """No noise, few tracks: every seed's best track is its own sim track, hit for hit."""
    wl = synth.workload(wl_name, n_events=3, tracks_lo=40, tracks_hi=40, noise_frac=0.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    f = oracle.find(g, b, sh, b.track_event[st])
    assert np.array_equal(f["hits"], b.track_hits[st])
    assert np.array_equal(f["n_hits"], b.track_nhits[st])


@pytest.mark.parametrize("wl_name", ["find", "hi_occ"])
def test_binned_and_brute_force_finding_agree(wl_name):
    wl = synth.workload(wl_name, n_events=2, tracks_lo=60, tracks_hi=60, noise_frac=2.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    a = oracle.find(g, b, sh, ev)
    c = oracle.find(g, b, sh, ev, brute_force=True)
    for k in ("hits", "n_hits", "status"):
        assert np.array_equal(a[k], c[k])
    assert np.array_equal(a["chi2"], c["chi2"])


@pytest.mark.parametrize("wl_name", ["find", "hi_occ"])
def test_window_counters_are_ordered(wl_name):
    """The windows limited to the phi sub-bins they touch hold every hit that passes the cut and
    no more hits than the windows' whole bins: passing <= sub-bin window hits <= whole-bin hits."""
    wl = synth.workload(wl_name, n_events=2, tracks_lo=300, tracks_hi=300, noise_frac=1.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    c = oracle.find(g, b, sh, b.track_event[st])["counters"]
    n_prop, n_pass, n_upd, n_scan, n_win, n_mlp = (int(v) for v in c)
    assert n_mlp == 0  # plain finding evaluates no network
    n_window_pass = n_pass - 3 * len(st)  # the pass counter includes the three seed-hit updates
    assert 0 < n_window_pass <= n_win <= n_scan
    assert n_win < n_scan  # the sub-bins cut the scan on these windows


def test_steering_that_lists_the_crossing_order_equals_the_geometric_rule():
    """Region steering (Sec. 3.1) on the barrel + disk geometry, whose disks start beyond the barrel
    half-length: every region list holds the surfaces a track of that region can reach in the order
    it crosses them (endcap lists truncated to the barrel layers an endcap track can reach), so the
    steered finder must reproduce the geometric next-surface rule exactly."""
    wl = synth.workload("hi_occ", n_events=2, tracks_lo=150, tracks_hi=150)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    geo = oracle.find(g, b, sh, ev)
    steered = oracle.find(g, b, sh, ev, steering=synth.steering_tables(wl, 0.4, 1.8, endcap_barrels=3))
    for k in ("hits", "n_hits", "status"):
        assert np.array_equal(geo[k], steered[k])
    assert np.array_equal(geo["chi2"], steered["chi2"], equal_nan=True)
    # the seeds span the regions: third seed hits on barrels (|z|/rho below and above the barrel
    # edge) and on disks
    s3 = b.hit_surface[sh[:, 2]]
    types = np.array([wl.surfaces[s].type for s in s3])
    zr = np.abs(b.hits[sh[:, 2], 1]) / np.array([wl.surfaces[s].r_or_z for s in s3])
    assert (types == synth.DISK).any() and ((types == synth.BARREL) & (zr > 0.42)).any()
    assert ((types == synth.BARREL) & (zr < 0.40)).any()


def test_steering_list_without_a_layer_passes_it_over():
    """A barrel list without layer 7: the found tracks hold no hit of layer 7, count no miss for
    it, and on clean sparse events lose exactly that hit."""
    wl = synth.workload("find", n_events=1, tracks_lo=60, tracks_hi=60, noise_frac=0.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, ms=False)
    sh, st = b.seeds()
    ev = b.track_event[st]
    tab = synth.steering_tables(wl, 10.0, 20.0)
    tab["lists"] = [[s for s in lst if s != 7] for lst in tab["lists"]]
    full = oracle.find(g, b, sh, ev)
    cut = oracle.find(g, b, sh, ev, steering=tab)
    on7 = np.isin(cut["hits"], np.nonzero(b.hit_surface == 7)[0])
    assert not on7.any()
    assert np.array_equal(full["n_hits"] - 1, cut["n_hits"])
    for i in range(len(st)):
        a = [h for h in full["hits"][i] if h >= 0 and b.hit_surface[h] != 7]
        c = [h for h in cut["hits"][i] if h >= 0]
        assert a == c


def test_invalid_seeds_fail_without_touching_the_rest():
    """A seed with a missing hit id or an event outside the batch has status 1 and no hits; the
    result of every other seed is the same as without them."""
    wl = synth.workload("find", n_events=2, tracks_lo=300, tracks_hi=300)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st].astype(np.int32)
    g = oracle.Geometry(wl)
    ref = oracle.find(g, b, sh, ev)
    bad_sh, bad_ev = sh.copy(), ev.copy()
    bad_sh[0, 1] = -1
    bad_sh[1, 0] = len(b.hits)
    bad_ev[2] = b.n_events
    bad_ev[3] = -1
    r = oracle.find(g, b, bad_sh, bad_ev)
    assert r["status"][:4].tolist() == [1, 1, 1, 1]
    assert np.all(r["hits"][:4] == -1) and np.all(r["n_hits"][:4] == 0)
    assert np.array_equal(r["hits"][4:], ref["hits"][4:]) and np.array_equal(r["status"][4:], ref["status"][4:])
