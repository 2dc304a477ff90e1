"""Pins of the oracle's learned hit proposal (CPU only): backpropagation against central finite
differences, training that lowers the loss, the pruning wired into the beam search checked
against a plain loop over the oracle's single-step primitives, and the disk value of the z-variance
feature."""
import numpy as np
import pytest

import oracle
import synth


def _pairs(n_events=2, stride=10, seed=4):
    wl = synth.workload("learned", n_events=n_events, tracks_lo=1500, tracks_hi=3000, seed=seed)
    b = synth.generate(wl)
    g = oracle.Geometry(wl)
    sh, st = b.seeds()
    sel = np.arange(0, len(st), stride)
    F, L = oracle.find_pairs(g, b, sh[sel], b.track_event[st][sel], st[sel])
    return F.astype(np.float64), L.astype(np.float64)


def test_backprop_matches_finite_differences():
    F, L = _pairs()
    mean, sd = F.mean(0), F.std(0)
    xs = (F[:64] - mean) / sd
    y = L[:64]
    w = synth.mlp_init(7).astype(np.float64)
    loss, g = oracle.mlp_loss_grad(w, xs, y)
    rng = np.random.default_rng(0)
    idx = np.concatenate([rng.choice(np.arange(0, 896), 20), rng.choice(np.arange(960, 5056), 40),
                          rng.choice(np.arange(5120, 5184), 10), [895, 900, 5100, 5184]])
    h = 1e-5
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (oracle.mlp_loss_grad(wp, xs, y)[0] - oracle.mlp_loss_grad(wm, xs, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3), (i, fd, g[i])
    # the logit of one sample by an explicit matrix chain
    W1, b1 = w[:896].reshape(64, 14), w[896:960]
    W2, b2 = w[960:5056].reshape(64, 64), w[5056:5120]
    W3, b3 = w[5120:5184], w[5184]
    z = W3 @ np.maximum(W2 @ np.maximum(W1 @ xs[3] + b1, 0) + b2, 0) + b3
    assert abs(oracle.mlp_forward(w, xs[3:4])[0] - z) < 1e-12


def test_adam_training_lowers_the_loss():
    F, L = _pairs(n_events=3, stride=8)
    mean, sd = F.mean(0), F.std(0)
    xs = (F - mean) / sd
    w = synth.mlp_init(11).astype(np.float64)
    m, v = np.zeros_like(w), np.zeros_like(w)
    rng = np.random.default_rng(1)
    first = oracle.mlp_loss_grad(w, xs, L)[0]
    for t in range(1, 201):
        b = rng.choice(len(L), 256, replace=False)
        _, g = oracle.mlp_loss_grad(w, xs[b], L[b])
        oracle.adam(w, g, m, v, t)
    last = oracle.mlp_loss_grad(w, xs, L)[0]
    assert last < 0.75 * first, (first, last)
    # the trained network ranks true continuations above other hits (area under the ROC curve:
    # the fraction of (true, other) pairs it orders correctly; 0.5 is chance)
    s = oracle.mlp_forward(w, xs)
    pos, neg = np.sort(s[L == 1]), s[L == 0]
    auc = np.searchsorted(pos, neg, side="right").sum() / (len(pos) * len(neg))
    auc = 1.0 - auc
    assert auc > 0.7, auc


def _mlp_for(F):
    return synth.mlp_init(3).astype(np.float64), F.mean(0), F.std(0) + 1e-9


def test_learned_with_large_top_n_is_plain_finding():
    wl = synth.workload("find", n_events=2, tracks_lo=400, tracks_hi=400, noise_frac=3.0)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    F, _ = oracle.find_pairs(g, b, sh, b.track_event[st], st)
    plain = oracle.find(g, b, sh, b.track_event[st])
    learned = oracle.find(g, b, sh, b.track_event[st], mlp=_mlp_for(F), top_n=1000)
    assert np.array_equal(plain["hits"], learned["hits"])
    assert learned["counters"][5] == 0  # no window has more passing hits than top_n


def test_learned_top1_matches_a_plain_loop():
    """K = 1, top_n = 1: at every step the kept hit is the passing hit of highest score."""
    import test_oracle_find as tf
    wl = synth.workload("find", n_events=2, tracks_lo=40, tracks_hi=40, noise_frac=80.0, seed=41)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    F, _ = oracle.find_pairs(g, b, sh, ev, st)
    mlp = _mlp_for(F)
    f = oracle.find(g, b, sh, ev, k_max=1, mlp=mlp, top_n=1)
    pruned = 0
    for i in range(len(st)):
        p, C, _ = tf._seed_fit(g, b, sh[i])
        hits, n_miss = list(sh[i]), 0
        while len(hits) < wl.lmax:
            e = tf._expand(g, b, wl, ev[i], p, C)
            if e is None:
                break
            surf, pp, CC, ids, c2 = e
            if len(ids) > 1:
                feats = np.array([oracle.pair_features(g, surf, pp, CC, b.hits[h]) for h in ids])
                sc = oracle.mlp_forward(mlp[0], (feats - mlp[1]) / mlp[2])
                order = sorted(range(len(ids)), key=lambda k: (-sc[k], ids[k]))
                ids, c2 = ids[order[:1]], c2[order[:1]]
                pruned += 1
            if len(ids):
                p, C, _ = oracle.update(g, pp, CC, surf, b.hits[ids[0]])
                hits.append(int(ids[0]))
            elif n_miss < wl.max_miss:
                p, C, n_miss = pp, CC, n_miss + 1
                hits.append(-1)
            else:
                break
        assert f["hits"][i].tolist() == hits + [-1] * (wl.lmax - len(hits)), i
    assert pruned > 10
    assert f["counters"][5] >= 2 * pruned  # every pruned window scores at least two hits


def test_disk_z_variance_feature_is_the_floor():
    """On a disk the state's z is fixed by the surface, so after propagation the z variance is
    zero (the covariance is projected onto the surface) and the log-variance feature equals its
    floor log(1e-12) to FP64 rounding; on a barrel it is a real variance, far above the floor."""
    wl = synth.workload("hi_occ")
    g = oracle.Geometry(wl)
    rng = np.random.default_rng(17)
    C0 = np.diag([1e-4, 1e-4, 1e-2, 1e-4, 1e-4, 1e-4])
    n_disk = n_barrel = 0
    for _ in range(200):
        th = rng.choice([rng.uniform(0.15, 0.5), rng.uniform(2.64, 2.99), rng.uniform(1.2, 1.9)])
        p0 = np.array([0.0, 0.0, 0.0, rng.choice([-1, 1]) * rng.uniform(0.1, 1.0), rng.uniform(-np.pi, np.pi), th])
        surf = (17 if th < 1.0 else 26) if abs(np.cos(th)) > 0.8 else 4
        r = oracle.propagate(g, p0, C0, surf)
        if r is None:
            continue
        p, C = r[0], r[1]
        hit = (np.arctan2(p[1], p[0]) + 1e-3, (np.hypot(p[0], p[1]) if surf != 4 else p[2]) + 0.05)
        f = oracle.pair_features(g, surf, p, C, hit)
        if surf == 4:
            n_barrel += 1
            assert f[8] > np.log(1e-12) + 10
        else:
            n_disk += 1
            assert abs(C[2, 2]) < 1e-15
            assert abs(f[8] - np.log(1e-12)) < 1e-3
        assert np.allclose(f[:6], p) and np.allclose(f[6:12], np.log(np.diag(C) + 1e-12))
    assert n_disk > 50 and n_barrel > 20


def _adam_steps(grads, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Weight trajectory of the oracle's Adam under a sequence of gradient vectors."""
    n = oracle.MLP_NPARAMS
    w = np.zeros(n)
    m, v = np.zeros(n), np.zeros(n)
    out = []
    for t, g in enumerate(grads, start=1):
        before = w.copy()
        oracle.adam(w, np.broadcast_to(g, (n,)).astype(np.float64).copy(), m, v, t, lr, b1, b2, eps)
        out.append(w - before)
    return out


def test_adam_first_step_is_lr_times_sign():
    """Kingma and Ba: after bias correction the first moments are m_hat = g and v_hat = g^2, so
    step 1 moves every weight by -lr g / (|g| + eps), i.e. lr against the sign of the gradient
    whatever its size (swapped moments would move by |g|-proportional steps)."""
    rng = np.random.default_rng(3)
    g = rng.choice([-1, 1], oracle.MLP_NPARAMS) * 10.0 ** rng.uniform(-3, 2, oracle.MLP_NPARAMS)
    (d,) = _adam_steps([g], lr=1e-3, eps=1e-8)
    assert np.allclose(d, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(np.abs(d), 1e-3, rtol=1e-5)


def test_adam_constant_gradient_keeps_a_step_of_lr():
    """With a constant gradient both bias-corrected moments are exact at every step (m_hat = g,
    v_hat = g^2), so the step stays lr: a correction by 1 - beta instead of 1 - beta^t would give
    1.9 lr at step 2."""
    g = np.full(oracle.MLP_NPARAMS, 0.37)
    steps = _adam_steps([g] * 25, lr=2e-3)
    for d in steps:
        assert np.allclose(d, -2e-3 * 0.37 / (0.37 + 1e-8), rtol=1e-9, atol=0)


def test_adam_two_steps_by_hand():
    """g1 = +1 then g2 = -1 (beta1 = 0.9, beta2 = 0.999): m2 = 0.9 * 0.1 - 0.1 = -0.01,
    1 - beta1^2 = 0.19, so m_hat = -1/19; v2 = 0.999 * 0.001 + 0.001 = 0.001999 = 1 - beta2^2,
    so v_hat = 1. The second step is +lr/19 (up to eps)."""
    d1, d2 = _adam_steps([1.0, -1.0], lr=1e-2, eps=1e-8)
    assert np.allclose(d1, -1e-2, rtol=1e-7)
    assert np.allclose(d2, 1e-2 / 19.0, rtol=1e-7)


def test_pull_features_of_true_hits_have_unit_width():
    """The last two features are the residuals over the square roots of the innovation variances
    (pulls). Along the true hit sequence of scattering-free tracks (predicted state from the hits
    before, as the fit makes it), the pulls of the next true hit have mean 0 and width 1: a
    division by S instead of sqrt(S), or a swapped residual, would not. The first surface after
    the seed is left out: the prior is centred on the seed made from hits 1-3, which changes the
    spread there."""
    wl = synth.workload("fit_small", n_events=1, tracks_lo=2500, tracks_hi=2500, seed=9)
    b = synth.generate(wl)
    g = oracle.Geometry(wl)
    pulls = []
    for t in range(b.n_tracks):
        ids = b.track_hits[t]
        ids = ids[ids >= 0]
        st = oracle.seed(g, b.hits, b.hit_surface, ids[:3])
        if st is None:
            continue
        p, C = st
        for k, h in enumerate(ids):
            surf = int(b.hit_surface[h])
            if k > 0:
                r = oracle.propagate(g, p, C, surf)
                assert r is not None
                p, C = r[0], r[1]
                if k >= 4:
                    pulls.append(oracle.pair_features(g, surf, p, C, b.hits[h])[12:])
            p, C, _ = oracle.update(g, p, C, surf, b.hits[h])
    x = np.array(pulls)
    assert len(x) > 10000
    assert np.all(np.abs(x.mean(0)) < 0.03), x.mean(0)
    assert np.all(np.abs(x.std(0) - 1.0) < 0.03), x.std(0)


def test_score_margin_limits_reduce_to_the_top_n_rule():
    """The score-margin rule at its limits: a margin larger than any score gap keeps the top_n of
    every window (the top_n rule, though windows of 2..top_n passing hits are now scored too); a
    vanishing margin keeps only the best-scoring hit (the top 1 rule, score ties having probability
    zero)."""
    wl = synth.workload("find", n_events=2, tracks_lo=400, tracks_hi=400, noise_frac=3.0, seed=43)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    F, _ = oracle.find_pairs(g, b, sh, ev, st)
    mlp = _mlp_for(F)
    top2 = oracle.find(g, b, sh, ev, mlp=mlp, top_n=2)
    wide = oracle.find(g, b, sh, ev, mlp=mlp, top_n=2, score_margin=1e9)
    assert np.array_equal(top2["hits"], wide["hits"])
    assert wide["counters"][5] > top2["counters"][5]  # windows of two passing hits are scored too
    top1 = oracle.find(g, b, sh, ev, mlp=mlp, top_n=1)
    narrow = oracle.find(g, b, sh, ev, mlp=mlp, top_n=2, score_margin=1e-12)
    assert np.array_equal(top1["hits"], narrow["hits"])
    assert not np.array_equal(top1["hits"], top2["hits"])


def test_score_margin_matches_a_plain_loop():
    """K = 1, top_n = 3, margin 0.7: at every step the kept hits are those among the three best
    scoring passing hits that score within 0.7 of the best, and the surviving child is the kept hit
    of lowest chi2."""
    import test_oracle_find as tf
    wl = synth.workload("find", n_events=2, tracks_lo=40, tracks_hi=40, noise_frac=80.0, seed=44)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    F, _ = oracle.find_pairs(g, b, sh, ev, st)
    mlp = _mlp_for(F)
    margin = 0.7
    f = oracle.find(g, b, sh, ev, k_max=1, mlp=mlp, top_n=3, score_margin=margin)
    multi = 0
    for i in range(len(st)):
        p, C, _ = tf._seed_fit(g, b, sh[i])
        hits, n_miss = list(sh[i]), 0
        while len(hits) < wl.lmax:
            e = tf._expand(g, b, wl, ev[i], p, C)
            if e is None:
                break
            surf, pp, CC, ids, c2 = e
            if len(ids) > 1:
                feats = np.array([oracle.pair_features(g, surf, pp, CC, b.hits[h]) for h in ids])
                sc = oracle.mlp_forward(mlp[0], (feats - mlp[1]) / mlp[2])
                order = sorted(range(len(ids)), key=lambda k: (-sc[k], ids[k]))[:3]
                keep = [k for k in order if sc[k] >= sc[order[0]] - margin]
                multi += len(keep) > 1
                ids, c2 = ids[keep], c2[keep]
            if len(ids):
                best = sorted(range(len(ids)), key=lambda k: (c2[k], ids[k]))[0]
                p, C, _ = oracle.update(g, pp, CC, surf, b.hits[ids[best]])
                hits.append(int(ids[best]))
            elif n_miss < wl.max_miss:
                p, C, n_miss = pp, CC, n_miss + 1
                hits.append(-1)
            else:
                break
        assert f["hits"][i].tolist() == hits + [-1] * (wl.lmax - len(hits)), i
    assert multi > 5  # the margin kept several hits in some windows


def test_window_ranking_with_a_top_n_above_every_window_is_plain_finding():
    """Ranking the window before the chi2 cut keeps every hit of a window that holds at most top_n:
    with top_n above any window's size the cut alone decides, as in plain finding."""
    wl = synth.workload("find", n_events=2, tracks_lo=300, tracks_hi=300, noise_frac=3.0, seed=45)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    F, _ = oracle.find_pairs(g, b, sh, ev, st)
    mlp = _mlp_for(F)
    plain = oracle.find(g, b, sh, ev)
    wide = oracle.find(g, b, sh, ev, mlp=mlp, top_n=100000, window=True)
    assert np.array_equal(plain["hits"], wide["hits"])
    assert wide["counters"][5] == 0
    narrow = oracle.find(g, b, sh, ev, mlp=mlp, top_n=2, window=True)
    assert narrow["counters"][5] > 0 and not np.array_equal(plain["hits"], narrow["hits"])


def test_window_ranking_with_a_margin_wider_than_any_gap_is_the_window_rule():
    """With a score margin the box is ranked from two hits on and only the top_n within the margin of
    the best face the cut: a margin wider than any score gap keeps all of the top_n, and a box of at
    most top_n hits is then kept whole, which is the window rule without a margin."""
    wl = synth.workload("find", n_events=2, tracks_lo=300, tracks_hi=300, noise_frac=3.0, seed=45)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    F, _ = oracle.find_pairs(g, b, sh, ev, st)
    mlp = _mlp_for(F)
    rule = oracle.find(g, b, sh, ev, mlp=mlp, top_n=2, window=True)
    wide = oracle.find(g, b, sh, ev, mlp=mlp, top_n=2, window=True, score_margin=1e9)
    assert np.array_equal(rule["hits"], wide["hits"])
    assert wide["counters"][5] > rule["counters"][5]  # boxes of two hits are scored too
    narrow = oracle.find(g, b, sh, ev, mlp=mlp, top_n=2, window=True, score_margin=0.5)
    assert not np.array_equal(rule["hits"], narrow["hits"])


@pytest.mark.parametrize("margin", [0.0, 1.0])
def test_window_ranking_matches_a_plain_loop(margin):
    """K = 1, top_n = 2, window ranking: at every step the box of the chi2 ellipse (both pulls within
    sqrt(cut)) is taken from every hit of the surface; when it holds more than two hits (with a score
    margin: two or more), only its two best-scoring hits (ties: lower id), with a margin only those
    scoring within it of the best, face the chi2 cut; the child is the kept passing hit of lowest
    chi2."""
    import test_oracle_find as tf
    wl = synth.workload("find", n_events=2, tracks_lo=40, tracks_hi=40, noise_frac=80.0, seed=46)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    sh, st = b.seeds()
    ev = b.track_event[st]
    F, _ = oracle.find_pairs(g, b, sh, ev, st)
    mlp = _mlp_for(F)
    cut = wl.chi2_cut
    f = oracle.find(g, b, sh, ev, k_max=1, mlp=mlp, top_n=2, window=True, score_margin=margin)
    ranked = cut_after_ranking = 0
    for i in range(len(st)):
        p, C, _ = tf._seed_fit(g, b, sh[i])
        hits, n_miss = list(sh[i]), 0
        while len(hits) < wl.lmax:
            surf, _ = oracle.next_surface(g, p)
            if surf < 0:
                break
            r = oracle.propagate(g, p, C, surf)
            if r is None:
                break
            pp, CC = r[0], r[1]
            ids, c2 = oracle.search(g, b, pp, CC, ev[i], surf, 1e30, brute=True)  # every hit of the surface
            feats = np.array([oracle.pair_features(g, surf, pp, CC, b.hits[h]) for h in ids]).reshape(-1, 14)
            inbox = (np.abs(feats[:, 12]) <= np.sqrt(cut)) & (np.abs(feats[:, 13]) <= np.sqrt(cut))
            bids, bc2, bf = ids[inbox], c2[inbox], feats[inbox]
            if len(bids) > (1 if margin > 0 else 2):
                ranked += 1
                sc = oracle.mlp_forward(mlp[0], (bf - mlp[1]) / mlp[2])
                top = sorted(range(len(bids)), key=lambda k: (-sc[k], bids[k]))[:2]
                if margin > 0:
                    top = [k for k in top if sc[k] >= sc[top[0]] - margin]
                keep = [k for k in top if bc2[k] < cut]
                cut_after_ranking += len(keep) < len(top)
                kids, kc2 = bids[keep], bc2[keep]
            else:
                kids, kc2 = bids[bc2 < cut], bc2[bc2 < cut]
            if len(kids):
                best = sorted(range(len(kids)), key=lambda k: (kc2[k], kids[k]))[0]
                p, C, _ = oracle.update(g, pp, CC, surf, b.hits[kids[best]])
                hits.append(int(kids[best]))
            elif n_miss < wl.max_miss:
                p, C, n_miss = pp, CC, n_miss + 1
                hits.append(-1)
            else:
                break
        assert f["hits"][i].tolist() == hits + [-1] * (wl.lmax - len(hits)), i
    print("ranked windows", ranked, "with a ranked hit cut", cut_after_ranking)
    assert ranked > 10 and cut_after_ranking >= 3  # the rule ranked windows, and the cut then removed ranked hits
