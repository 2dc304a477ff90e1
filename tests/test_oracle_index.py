"""Pins of the oracle's hit index and windowed hit search (CPU only).

The FP32 binning rule is recomputed with numpy float32 arithmetic (IEEE single, each operation
rounded on its own), the index is checked against numpy's stable argsort, and the binned search
is checked against brute force over every hit of the surface.
"""
import numpy as np
import pytest

import oracle
import synth


def _np_sub(wl, surf, phi, pb):
    """Phi sub-bin: fine = clamp(floor((phi + pi_f) * (float)(n_phi*8/2pi)), 0, n_phi*8 - 1) in
    float32, then clamp(fine - pb*8, 0, 7)."""
    s = wl.surfaces[surf]
    a = (np.asarray(phi, np.float32) + np.float32(np.pi)).astype(np.float32)
    a = (a * np.float32(s.n_phi * 8 / (2.0 * np.pi))).astype(np.float32)
    fine = np.clip(np.floor(a), -1, 1e8).astype(np.int64).clip(0, s.n_phi * 8 - 1)
    return np.clip(fine - pb * 8, 0, 7)


def _np_bins(wl, surf, phi, second):
    """phi-bin = clamp(floor((phi + pi_f) * (float)(n_phi/2pi)), 0, n_phi-1); second coordinate
    likewise with (float)(n_2nd / (hi_f - lo_f)); every operation in float32."""
    s = wl.surfaces[surf]
    pi_f = np.float32(np.pi)
    sphi = np.float32(s.n_phi / (2.0 * np.pi))
    lo = np.float32(s.lo)
    s2 = np.float32(s.n_2nd / (float(np.float32(s.hi)) - float(np.float32(s.lo))))
    a = (np.asarray(phi, np.float32) + pi_f).astype(np.float32)
    a = (a * sphi).astype(np.float32)
    b = (np.asarray(second, np.float32) - lo).astype(np.float32)
    b = (b * s2).astype(np.float32)
    pb = np.clip(np.floor(a), -1, 1e8).astype(np.int64).clip(0, s.n_phi - 1)
    zb = np.clip(np.floor(b), -1, 1e8).astype(np.int64).clip(0, s.n_2nd - 1)
    return pb, zb


def test_bin_rule_matches_float32_arithmetic():
    wl = synth.workload("hi_occ")
    g = oracle.Geometry(wl)
    rng = np.random.default_rng(0)
    edge_phi = np.array([-np.pi, np.nextafter(np.float32(np.pi), np.float32(0)), 0.0, np.float32(np.pi),
                         -np.float32(np.pi)], np.float32)
    for surf in (0, 5, 16, 17, 30):
        s = wl.surfaces[surf]
        phi = np.concatenate([rng.uniform(-np.pi, np.pi, 3000).astype(np.float32), edge_phi])
        # bin edges themselves, and values just around them
        k = np.arange(s.n_phi + 1)
        e = (k / (s.n_phi / (2 * np.pi)) - np.pi).astype(np.float32)
        phi = np.concatenate([phi, e, np.nextafter(e, np.float32(-10)), np.nextafter(e, np.float32(10))])
        sec = rng.uniform(s.lo - 1, s.hi + 1, phi.size).astype(np.float32)
        pb, zb = _np_bins(wl, surf, phi, sec)
        for i in range(phi.size):
            assert oracle.bin_of(g, surf, phi[i], sec[i]) == (pb[i], zb[i]), (surf, phi[i], sec[i])


@pytest.mark.parametrize("wl_name", ["find", "hi_occ"])
def test_index_is_sort_by_bin_subbin_id(wl_name):
    wl = synth.workload(wl_name, n_events=2, tracks_lo=400, tracks_hi=600)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    off, sh, si, sub = oracle.build_index(g, b.hits, b.slab_offsets, b.n_events, with_sub=True)
    ns = b.n_surf
    for sl in range(b.n_events * ns):
        surf = sl % ns
        s = wl.surfaces[surf]
        nbs = s.n_phi * s.n_2nd
        h0, h1 = b.slab_offsets[sl], b.slab_offsets[sl + 1]
        pb, zb = _np_bins(wl, surf, b.hits[h0:h1, 0], b.hits[h0:h1, 1])
        key = pb * s.n_2nd + zb
        sb = _np_sub(wl, surf, b.hits[h0:h1, 0], pb)
        order = np.lexsort((np.arange(h1 - h0), sb, key))
        assert np.array_equal(si[h0:h1], h0 + order)
        assert np.array_equal(sh[h0:h1], b.hits[h0 + order])
        counts = np.bincount(key, minlength=nbs)
        assert off[sl, 0] == h0
        assert np.array_equal(np.diff(off[sl, : nbs + 1]), counts)
        # sub-bin offsets: hits of each bin with sub-bin <= j
        per = np.zeros((nbs, 8), np.int64)
        np.add.at(per, (key, sb), 1)
        assert np.array_equal(sub[sl, :nbs].astype(np.int64), np.cumsum(per, axis=1))
        assert not sub[sl, nbs:].any()


def test_subbin_rule_is_monotone_within_a_bin():
    """Within a phi bin the sub-bin never decreases with phi (windows rely on it), including across
    the rounding of the fine index at the bin edges."""
    wl = synth.workload("find")
    g = oracle.Geometry(wl)
    phi = np.sort(np.concatenate([np.linspace(-np.pi, np.pi, 200001),
                                  (np.arange(65) * 2 * np.pi / 64 - np.pi)]).astype(np.float32))
    phi = np.unique(np.concatenate([phi, np.nextafter(phi, np.float32(-10)), np.nextafter(phi, np.float32(10))]))
    phi = phi[(phi >= -np.float32(np.pi)) & (phi <= np.float32(np.pi))]
    pb, _ = _np_bins(wl, 0, phi, np.zeros_like(phi))
    sb = _np_sub(wl, 0, phi, pb)
    same = pb[1:] == pb[:-1]
    assert (sb[1:][same] >= sb[:-1][same]).all()
    assert set(np.unique(sb)) == set(range(8))


def _candidate_states(b, g, rng, n):
    """Predicted states at random surfaces: true tracks propagated from their previous crossing,
    with covariances inflated at random so windows span from one bin to the whole surface."""
    out = []
    for _ in range(n):
        t = int(rng.integers(0, b.n_tracks))
        nh = b.track_nhits[t]
        k = int(rng.integers(0, nh - 1))
        A = rng.normal(size=(6, 6)) * 10 ** rng.uniform(-4, -1)
        C0 = A @ A.T + np.diag([1e-5, 1e-5, 1e-4, 1e-4, 1e-6, 1e-6]) * 10 ** rng.uniform(0, 9)
        r = oracle.propagate(g, b.truth_out[t, k], C0, b.track_surf[t, k + 1])
        if r is not None:
            out.append((b.track_event[t], b.track_surf[t, k + 1], r[0], r[1]))
    return out


@pytest.mark.parametrize("wl_name", ["find", "hi_occ"])
def test_binned_search_equals_brute_force(wl_name):
    """The window is the padded bounding box of the chi2 < cut ellipse, so the binned search
    returns exactly the hits brute force finds, for small and very wide windows, near phi = +-pi
    and at the z (or r) ends."""
    wl = synth.workload(wl_name, n_events=1, tracks_lo=120, tracks_hi=120, noise_frac=3.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, record_truth=True)
    rng = np.random.default_rng(1)
    n_nonempty = 0
    for ev, surf, p, C in _candidate_states(b, g, rng, 400):
        ib, cb = oracle.search(g, b, p, C, ev, surf, wl.chi2_cut, brute=False)
        iu, cu = oracle.search(g, b, p, C, ev, surf, wl.chi2_cut, brute=True)
        assert sorted(ib.tolist()) == sorted(iu.tolist())
        assert np.allclose(np.sort(cb), np.sort(cu), rtol=0, atol=0)
        n_nonempty += len(iu) > 0
    assert n_nonempty > 100
