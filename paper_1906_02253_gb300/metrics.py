"""Track-finding efficiency and fake rate (host-side validation of found tracks).

Follows the standalone validation of Sec. 4, adapted to these events: the denominator holds the
simulated tracks that leave 10 or more hits; the track found from a seed counts for the seed's
simulated track when it carries min(10, crossings - 1) hits or more and half or more of its
non-seed hits come from that track (seeds here have 3 hits, the paper's 4).
"""
from __future__ import annotations

import numpy as np


def efficiency(batch, seed_track, found_hits, found_nhits, min_hits: int = 10, match_frac: float = 0.5):
    """Returns (efficiency, fake_rate). found_hits is [n_seeds, lmax] (hit ids, -1 = none)."""
    seed_track = np.asarray(seed_track)
    fh = np.asarray(found_hits)
    nh = np.asarray(found_nhits)
    n_true = batch.track_nhits[seed_track]
    need = np.minimum(min_hits, n_true - 1)
    ext = fh[:, 3:]
    valid = ext >= 0
    sim = batch.hit_sim[np.where(valid, ext, 0)]
    own = valid & (sim == seed_track[:, None])
    n_ext = valid.sum(axis=1)
    n_own = own.sum(axis=1)
    matched = (nh >= need) & (n_ext > 0) & (n_own >= match_frac * n_ext)
    ref = n_true >= min_hits
    eff = float(matched[ref].mean()) if ref.any() else float("nan")
    fake = float(1.0 - matched.mean()) if matched.size else float("nan")
    return eff, fake


def majority_sim(batch, found_hits, found_nhits, min_hits: int = 10, match_frac: float = 0.5, chunk: int = 32768):
    """Simulated track each found track belongs to, whatever its seed (-1: none): the one holding
    more than ``match_frac`` of the track's hits, for tracks with at least min(min_hits,
    crossings - 1) hits (hit-fraction matching, as in the paper's validation, Sec. 4)."""
    fh = np.asarray(found_hits)
    nh = np.asarray(found_nhits)
    out = np.full(len(fh), -1, np.int64)
    for a in range(0, len(fh), chunk):
        h = fh[a:a + chunk]
        valid = h >= 0
        sim = np.where(valid, batch.hit_sim[np.where(valid, h, 0)], -1)
        same = (sim[:, :, None] == sim[:, None, :]) & (sim[:, None, :] >= 0)
        cnt = np.where(sim >= 0, same.sum(axis=2), 0)
        best = cnt.argmax(axis=1)
        rows = np.arange(len(h))
        top, s = cnt[rows, best], sim[rows, best]
        need = np.minimum(min_hits, batch.track_nhits[np.maximum(s, 0)] - 1)
        ok = (top > match_frac * valid.sum(axis=1)) & (s >= 0) & (nh[a:a + chunk] >= need)
        out[a:a + chunk] = np.where(ok, s, -1)
    return out


def track_rates(batch, seed_track, found_hits, found_nhits, keep=None, min_hits: int = 10):
    """(efficiency, duplicate rate, fake rate) per simulated track when several seeds may come from
    one particle. Reference tracks: simulated tracks with >= min_hits hits and a seed. Efficiency:
    reference tracks with at least one kept track matched to them (majority_sim); duplicate rate:
    those with two or more; fake rate: kept tracks with hits matched to no simulated track."""
    st = np.asarray(seed_track)
    sim = majority_sim(batch, found_hits, found_nhits, min_hits)
    kept = np.ones(len(st), bool) if keep is None else np.asarray(keep) != 0
    kept &= np.asarray(found_nhits) > 0
    m = kept & (sim >= 0)
    counts = np.bincount(sim[m], minlength=batch.n_tracks)
    ref = np.zeros(batch.n_tracks, bool)
    ref[st] = True
    ref &= batch.track_nhits >= min_hits
    eff = float((counts[ref] >= 1).mean()) if ref.any() else float("nan")
    dup = float((counts[ref] >= 2).mean()) if ref.any() else float("nan")
    fake = float(1.0 - m.sum() / kept.sum()) if kept.any() else float("nan")
    return eff, dup, fake
