"""Train the learned hit-proposal network and store it for the finder (run on a GPU machine).

Training pairs come from the FP64 oracle's plain finding on 200 generated events of the learned
workload (the 100-event workload's geometry and occupancy, seed 4): every (candidate, hit) pair
that passes the chi2 cut, labelled 1 when the hit belongs to the seed's simulated track. Seeds are
subsampled (every 10th) to keep the pair count near 14 million. The network starts from the input generator's
He initialisation and is trained by the library's kernels (kf_mlp_loss_grad, kf_mlp_adam); the
host only shuffles minibatches. One pair in ten is held out to measure the ranking quality.

    python tests/train_learned_proposal.py [--out paper_1906_02253_gb300/data/mlp_learned.npz]
    python tests/train_learned_proposal.py --workload hi_occ --stride 20 \
        --out paper_1906_02253_gb300/data/mlp_hi_occ.npz
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def auc_of(scores, labels):
    pos, neg = np.sort(scores[labels == 1]), scores[labels == 0]
    return 1.0 - np.searchsorted(pos, neg, side="right").sum() / (len(pos) * len(neg))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(ROOT, "paper_1906_02253_gb300", "data", "mlp_learned.npz"))
    ap.add_argument("--workload", default="learned", help="learned (barrel) or hi_occ (barrel + disks)")
    ap.add_argument("--events", type=int, default=200)
    ap.add_argument("--stride", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-halving", type=int, default=4)
    ap.add_argument("--init-seed", type=int, default=2024)
    args = ap.parse_args()

    import __graft_entry__ as ge
    ge.build()
    import paper_1906_02253_gb300 as kf

    t0 = time.time()
    wl = synth.workload(args.workload, n_events=args.events)
    b = synth.generate(wl)
    g = oracle.Geometry(wl)
    sh, st = b.seeds()
    sel = np.arange(0, len(st), args.stride)
    F, L = oracle.find_pairs(g, b, sh[sel], b.track_event[st][sel], st[sel], cap=20_000_000)
    t_pairs = time.time() - t0
    rng = np.random.default_rng(1)
    hold = rng.random(len(L)) < 0.1
    Ftr, Ltr, Fte, Lte = F[~hold], L[~hold], F[hold], L[hold]
    mean = Ftr.mean(0).astype(np.float32)
    sd = (Ftr.std(0) + 1e-6).astype(np.float32)
    params = kf.mlp_buffer(synth.mlp_init(args.init_seed), mean, sd)
    t1 = time.time()
    hist = kf.mlp_train(params, torch.from_numpy(Ftr).cuda(), torch.from_numpy(Ltr).cuda(), epochs=args.epochs,
                        batch=args.batch, lr=args.lr, log=print, lr_halving=args.lr_halving)
    torch.cuda.synchronize()
    t_train = time.time() - t1
    sc = kf.mlp_forward(params, torch.from_numpy(Fte).cuda()).cpu().numpy()
    auc = auc_of(sc, Lte)
    w = params.cpu().numpy()
    info = dict(workload=args.workload, events=args.events, seed=wl.seed, seed_stride=args.stride, pairs=int(len(L)), lr_halving=args.lr_halving,
                positive_fraction=float(L.mean()), held_out=int(hold.sum()), held_out_auc=float(auc),
                loss_per_epoch=hist, epochs=args.epochs, batch=args.batch, lr=args.lr, init_seed=args.init_seed,
                seconds_pairs=t_pairs, seconds_train=t_train)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    np.savez(args.out, weights=w[: kf.MLP_PARAMS], mean=mean, sd=sd, info=json.dumps(info))
    print(json.dumps(info))


if __name__ == "__main__":
    main()
