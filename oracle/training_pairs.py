"""Labelled training pairs of the learned hit proposal, from the oracle's own finding.

TEST INFRASTRUCTURE (part of the oracle): the network is trained on what the FP64 oracle's plain
finding sees on generated events. Every (candidate, hit) pair that passes the chi2 cut in the
oracle's beam search from the seeds of a workload's events (every `stride`-th seed) becomes one
row of 14 features (the oracle's pair features) with label 1 when the hit belongs to the seed's
simulated track, else 0. The pairs file is the input of the library's training step:

    python -m oracle.training_pairs --workload learned --events 200 --stride 10 --out pairs_learned.npz
    python -m paper_1906_02253_gb300.train pairs_learned.npz paper_1906_02253_gb300/data/mlp_learned.npz

    python -m oracle.training_pairs --workload hi_occ --events 200 --stride 20 --out pairs_hi_occ.npz
    python -m paper_1906_02253_gb300.train pairs_hi_occ.npz paper_1906_02253_gb300/data/mlp_hi_occ.npz
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def make_pairs(workload: str, events: int, stride: int, cap: int = 20_000_000):
    """(features [n, 14] float32, labels [n] float32, metadata) of the workload's generated events."""
    t0 = time.time()
    wl = synth.workload(workload, n_events=events)
    b = synth.generate(wl)
    sh, st = b.seeds()
    sel = np.arange(0, len(st), stride)
    F, L = oracle.find_pairs(oracle.Geometry(wl), b, sh[sel], b.track_event[st][sel], st[sel], cap=cap)
    meta = dict(workload=workload, events=events, seed=wl.seed, seed_stride=stride, pairs=int(len(L)),
                positive_fraction=float(L.mean()) if len(L) else 0.0, seconds_pairs=time.time() - t0)
    return F, L, meta


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="learned", help="learned (barrel) or hi_occ (barrel + disks)")
    ap.add_argument("--events", type=int, default=200)
    ap.add_argument("--stride", type=int, default=10)
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    F, L, meta = make_pairs(args.workload, args.events, args.stride)
    np.savez(args.out, features=F, labels=L, meta=json.dumps(meta))
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
