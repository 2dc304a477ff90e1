"""Efficiency definition and the paper's stated constants (CPU only)."""
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


def test_workloads_use_the_papers_field():
    g = _golden()
    for wl in synth.WORKLOADS.values():
        assert wl.bz == g["bz_tesla"]


def test_efficiency_definition_on_hand_made_tracks():
    """Tiny hand-made event: hit ids 0..19 belong to sim track 0 and 20..39 to sim track 1;
    40.. are noise. Checks the hit-count threshold and the 50% rule (Sec. 4)."""
    g = _golden()
    wl = synth.workload("find")

    class B:
        pass

    b = B()
    b.track_nhits = np.array([17, 17])
    b.hit_sim = np.array([0] * 20 + [1] * 20 + [-1] * 20)
    n = 4
    seed_track = np.array([0, 0, 1, 1])
    hits = -np.ones((n, wl.lmax), np.int32)
    hits[0, :12] = np.arange(12)                                     # all own hits: matched
    hits[1, :3] = [0, 1, 2]; hits[1, 3:12] = [3, 4, 5, 6] + [40, 41, 42, 43, 44]  # 4 of 9 own: fake
    hits[2, :3] = [20, 21, 22]; hits[2, 3:11] = [23, 24, 25, 26, 40, 41, 42, 43]  # 4 of 8 own: matched
    hits[3, :3] = [20, 21, 22]; hits[3, 3:9] = [23, 24, 25, 26, 27, 28]          # 9 hits: too short
    nh = (hits >= 0).sum(1)
    eff, fake, matched = oracle.efficiency(b, seed_track, hits, nh, min_hits=int(g["min_found_hits"]),
                                           match_frac=g["match_fraction"])
    assert matched.tolist() == [True, False, True, False]
    assert eff == 0.5 and fake == 0.5


def test_clean_events_are_fully_efficient():
    wl = synth.workload("find", n_events=2, tracks_lo=50, tracks_hi=50, noise_frac=0.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    f = oracle.find(g, b, sh, b.track_event[st])
    eff, fake, _ = oracle.efficiency(b, st, f["hits"], f["n_hits"])
    assert eff == 1.0 and fake == 0.0


def test_package_efficiency_matches_oracle_definition():
    """The package's vectorised efficiency (used by the benchmark) equals the oracle's loop."""
    from paper_1906_02253_gb300 import metrics
    wl = synth.workload("find", n_events=2, tracks_lo=300, tracks_hi=300, noise_frac=3.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    f = oracle.find(g, b, sh, b.track_event[st], k_max=1)
    e1, f1, _ = oracle.efficiency(b, st, f["hits"], f["n_hits"])
    e2, f2 = metrics.efficiency(b, st, f["hits"], f["n_hits"])
    assert e1 == e2 and f1 == f2
    assert 0.9 < e1 <= 1.0
