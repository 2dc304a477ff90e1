"""Training of the learned hit-proposal network by the library's own kernels.

Input: a file of labelled pairs (features [n, 14], labels [n]; the pairs the oracle's finding
produces on generated events, see oracle/training_pairs.py). One pair in ten (a fixed seeded choice)
is held out; the feature normaliser is the mean and standard deviation of the rest; the network
starts from the input generator's He initialisation and is trained with minibatch Adam, every step
in the library's kernels (kf_mlp_loss_grad, kf_mlp_adam); the host only shuffles minibatches. The
held-out area under the ROC curve measures the ranking. Output: the weights, the normaliser and a
record of the run, the file the finder's learned proposal loads.

    python -m paper_1906_02253_gb300.train pairs.npz paper_1906_02253_gb300/data/mlp_learned.npz
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch


def auc_of(scores, labels) -> float:
    """Area under the ROC curve: the fraction of (positive, negative) pairs ranked correctly."""
    pos, neg = np.sort(scores[labels == 1]), scores[labels == 0]
    return float(1.0 - np.searchsorted(pos, neg, side="right").sum() / (len(pos) * len(neg)))


def train(features, labels, epochs: int = 12, batch: int = 4096, lr: float = 2e-3, lr_halving: int = 4,
          init_seed: int = 2024, log=None):
    """Train on (features, labels) arrays; returns (weights, mean, sd, record)."""
    import synth
    import paper_1906_02253_gb300 as kf
    rng = np.random.default_rng(1)
    hold = rng.random(len(labels)) < 0.1
    ftr, ltr, fte, lte = features[~hold], labels[~hold], features[hold], labels[hold]
    mean = ftr.mean(0).astype(np.float32)
    sd = (ftr.std(0) + 1e-6).astype(np.float32)
    params = kf.mlp_buffer(synth.mlp_init(init_seed), mean, sd)
    t0 = time.time()
    hist = kf.mlp_train(params, torch.from_numpy(np.ascontiguousarray(ftr)).cuda(),
                        torch.from_numpy(np.ascontiguousarray(ltr)).cuda(), epochs=epochs, batch=batch, lr=lr,
                        log=log, lr_halving=lr_halving)
    torch.cuda.synchronize()
    seconds = time.time() - t0
    sc = kf.mlp_forward(params, torch.from_numpy(np.ascontiguousarray(fte)).cuda()).cpu().numpy()
    rec = dict(held_out=int(hold.sum()), held_out_auc=auc_of(sc, lte), loss_per_epoch=hist, epochs=epochs,
               batch=batch, lr=lr, lr_halving=lr_halving, init_seed=init_seed, seconds_train=seconds)
    return params.cpu().numpy()[: kf.MLP_PARAMS], mean, sd, rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("pairs")
    ap.add_argument("out")
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--lr-halving", type=int, default=4)
    ap.add_argument("--init-seed", type=int, default=2024)
    args = ap.parse_args()
    import paper_1906_02253_gb300 as kf
    kf.load_library()
    z = np.load(args.pairs)
    meta = json.loads(str(z["meta"]))
    w, mean, sd, rec = train(z["features"], z["labels"], args.epochs, args.batch, args.lr, args.lr_halving,
                             args.init_seed, log=print)
    info = dict(meta, **rec)
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    np.savez(args.out, weights=w, mean=mean, sd=sd, info=json.dumps(info))
    print(json.dumps(info))


if __name__ == "__main__":
    main()
