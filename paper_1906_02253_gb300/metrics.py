"""Track-finding efficiency and fake rate (host-side validation of found tracks).

Adapted from the paper's standalone validation (Sec. 4): reference tracks are simulated tracks
with at least 10 hits; a seed's found track is matched to the seed's simulated track when it has
at least min(10, crossings - 1) hits and at least 50% of its hits beyond the three seed hits
belong to that track (the paper's seeds have 4 hits; ours have 3).
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
