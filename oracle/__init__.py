"""FP64 CPU oracle for Kalman-filter track fitting and finding (ctypes over ``kf_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg are the only callers. It shares no code with the CUDA path. Plain, slow, obviously
correct: full 6x6 FP64 matrices, textbook helix/Kalman formulas (the paper, Sec. 1-2, names the
traditional Kalman filter and prints no formulas), an FP32 hit-binning rule evaluated with every
operation rounded separately, and a beam search that keeps the best K candidates per seed.

Also: region steering, the r-z material map with energy loss, the parametrised field, seed
cleaning and duplicate removal, and the learned proposal's network, as the paper's options.

Parity unpinned: the prior widths, the candidate ranking key, the barrel half-lengths and disk
extents, the efficiency definition, the cleaning and removal cuts and the synthetic material and
field values are readings chosen where the paper is silent; they are fixed here, not checked
against numbers the paper prints (it prints none).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libkforacle.so")
_lib = None
_lock = threading.Lock()

K_CURV = 0.00299792458  # GeV / (T cm)


def build_native(force: bool = False) -> str:
    """Compile the oracle. ``-ffp-contract=off`` keeps every FP32 binning operation separately
    rounded (no fused multiply-add), which the bit-exact binning rule requires."""
    src = os.path.join(_HERE, "kf_oracle.cpp")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, src, "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrSurface(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("r_or_z", ctypes.c_float), ("lo", ctypes.c_float),
                ("hi", ctypes.c_float), ("x_over_x0", ctypes.c_float), ("n_phi", ctypes.c_int),
                ("n_2nd", ctypes.c_int)]


class OrGeom(ctypes.Structure):
    _fields_ = [("bz", ctypes.c_float), ("n_surf", ctypes.c_int), ("surf", ctypes.POINTER(OrSurface)),
                ("sigma_rphi", ctypes.c_float), ("sigma_2nd", ctypes.c_float), ("prior", ctypes.c_float * 5),
                ("ms_off", ctypes.c_int), ("material", ctypes.c_void_p), ("eloss", ctypes.c_float),
                ("mass", ctypes.c_float), ("field_z2", ctypes.c_float), ("field_r2", ctypes.c_float)]


class OrFindParams(ctypes.Structure):
    _fields_ = [("chi2_cut", ctypes.c_float), ("k_max", ctypes.c_int), ("max_miss", ctypes.c_int),
                ("brute_force", ctypes.c_int)]


_P = ctypes.c_void_p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_native())
            G = ctypes.POINTER(OrGeom)
            lib.or_propagate.restype = ctypes.c_int
            lib.or_propagate.argtypes = [G, _P, _P, ctypes.c_int, _P, _P, _P, _P]
            lib.or_helix_at.argtypes = [G, _P, ctypes.c_double, _P]
            lib.or_seed.restype = ctypes.c_int
            lib.or_seed.argtypes = [G, _P, _P, _P, _P, _P]
            lib.or_fit.argtypes = [G, _P, _P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                   _P, _P, _P, _P, _P, _P, _P]
            lib.or_index_bins.restype = ctypes.c_int
            lib.or_index_bins.argtypes = [G]
            lib.or_build_index.argtypes = [G, _P, _P, ctypes.c_int, _P, _P, _P, _P]
            lib.or_bin_of.argtypes = [G, ctypes.c_int, ctypes.c_float, ctypes.c_float, _P, _P]
            lib.or_search.restype = ctypes.c_int
            lib.or_search.argtypes = [G, _P, _P, _P, ctypes.c_int, _P, _P, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_float, ctypes.c_int, ctypes.c_int, _P, _P]
            lib.or_update.restype = ctypes.c_double
            lib.or_update.argtypes = [G, _P, _P, ctypes.c_int, ctypes.c_float, ctypes.c_float, _P, _P]
            lib.or_next_surface.restype = ctypes.c_int
            lib.or_next_surface.argtypes = [G, _P, _P]
            lib.or_find.argtypes = [G, _P, _P, _P, ctypes.c_int, _P, _P, ctypes.c_longlong, ctypes.c_int,
                                    ctypes.POINTER(OrFindParams), ctypes.c_int, _P, _P, _P, _P, _P, _P, _P,
                                    _P, _P, _P, ctypes.c_int, ctypes.POINTER(OrSteering), ctypes.c_double,
                                    ctypes.c_int]
            lib.or_seed_params.argtypes = [G, _P, _P, _P, ctypes.c_longlong, _P]
            lib.or_clean_seeds.argtypes = [_P, _P, _P, ctypes.c_longlong, ctypes.c_double, ctypes.c_double, _P]
            lib.or_remove_duplicates.argtypes = [_P, _P, _P, _P, _P, _P, ctypes.c_longlong, ctypes.c_int,
                                                 ctypes.c_double, ctypes.c_double, _P]
            lib.or_mlp_nparams.restype = ctypes.c_int
            lib.or_find_pairs.restype = ctypes.c_longlong
            lib.or_find_pairs.argtypes = [G, _P, _P, _P, ctypes.c_int, _P, _P, _P, _P, ctypes.c_longlong,
                                          ctypes.c_int, ctypes.POINTER(OrFindParams), ctypes.c_int,
                                          ctypes.c_longlong, _P, _P]
            lib.or_mlp_forward.argtypes = [_P, _P, ctypes.c_longlong, _P]
            lib.or_pair_features.argtypes = [G, ctypes.c_int, _P, _P, ctypes.c_float, ctypes.c_float, _P]
            lib.or_mlp_loss_grad.restype = ctypes.c_double
            lib.or_mlp_loss_grad.argtypes = [_P, _P, _P, ctypes.c_longlong, _P]
            lib.or_adam.argtypes = [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double]
            _lib = lib
    return _lib


class Geometry:
    """Oracle-side geometry built from a ``synth.Workload`` (FP32 values are canonical)."""

    def __init__(self, wl):
        self.wl = wl
        n = len(wl.surfaces)
        self._surf = (OrSurface * n)()
        for i, s in enumerate(wl.surfaces):
            self._surf[i] = OrSurface(s.type, s.r_or_z, s.lo, s.hi, s.x_over_x0, s.n_phi, s.n_2nd)
        mat = getattr(wl, "material", None)
        self._mat = None if mat is None else np.ascontiguousarray(mat, dtype=np.float32)
        self.g = OrGeom(wl.bz, n, ctypes.cast(self._surf, ctypes.POINTER(OrSurface)), wl.sigma_rphi,
                        wl.sigma_2nd, (ctypes.c_float * 5)(*wl.prior), int(not wl.ms_on),
                        None if self._mat is None else self._mat.ctypes.data, getattr(wl, "eloss", 0.0),
                        getattr(wl, "mass", 0.13957), getattr(wl, "field_z2", 0.0), getattr(wl, "field_r2", 0.0))

    @property
    def ref(self):
        return ctypes.byref(self.g)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def propagate(geom: Geometry, p, C, surf: int):
    """Propagate state ``p`` (6) with covariance ``C`` (6x6) to surface ``surf``.
    Returns (p', C', J, s) or None if the surface is not reached."""
    lib = _load()
    p = _c(p, np.float64)
    C = _c(C if C is not None else np.zeros((6, 6)), np.float64)
    po, Co, J = np.empty(6), np.empty((6, 6)), np.empty((6, 6))
    s = ctypes.c_double()
    rc = lib.or_propagate(geom.ref, p.ctypes.data, C.ctypes.data, surf, po.ctypes.data, Co.ctypes.data,
                          J.ctypes.data, ctypes.addressof(s))
    return None if rc != 0 else (po, Co, J, s.value)


def helix_at(geom: Geometry, p, s: float):
    lib = _load()
    p = _c(p, np.float64)
    out = np.empty(6)
    lib.or_helix_at(geom.ref, p.ctypes.data, float(s), out.ctypes.data)
    return out


def seed(geom: Geometry, hits, hit_surface, ids):
    lib = _load()
    hits = _c(hits, np.float32)
    hs = _c(hit_surface, np.int32)
    ids = _c(ids, np.int32)
    p, C = np.empty(6), np.empty((6, 6))
    rc = lib.or_seed(geom.ref, hits.ctypes.data, hs.ctypes.data, ids.ctypes.data, p.ctypes.data, C.ctypes.data)
    return None if rc != 0 else (p, C)


def fit(geom: Geometry, hits, hit_surface, track_hits, n_threads: int = 0, per_hit: bool = False):
    """Fit every track over its known hit sequence (``track_hits`` [n, lmax], -1 padded).
    Returns dict with p [n,6], cov [n,21] (packed upper triangle), chi2, ndof, status and,
    with ``per_hit``, hit_chi2 [n,lmax] and hit_pull [n,lmax,2]."""
    lib = _load()
    hits = _c(hits, np.float32)
    hs = _c(hit_surface, np.int32)
    th = _c(track_hits, np.int32)
    n, lmax = th.shape
    out = dict(p=np.empty((n, 6)), cov=np.empty((n, 21)), chi2=np.empty(n), ndof=np.empty(n, np.int32),
               status=np.empty(n, np.int32))
    hc = np.empty((n, lmax)) if per_hit else None
    hp = np.empty((n, lmax, 2)) if per_hit else None
    lib.or_fit(geom.ref, hits.ctypes.data, hs.ctypes.data, th.ctypes.data, n, lmax, n_threads,
               out["p"].ctypes.data, out["cov"].ctypes.data, out["chi2"].ctypes.data, out["ndof"].ctypes.data,
               out["status"].ctypes.data, hc.ctypes.data if per_hit else None, hp.ctypes.data if per_hit else None)
    if per_hit:
        out["hit_chi2"] = hc
        out["hit_pull"] = hp
    return out


PHI_SUB = 8  # phi sub-bins per phi bin


def build_index(geom: Geometry, hits, slab_offsets, n_events: int, with_sub: bool = False):
    """Returns (bin_off [n_events*n_surf, nb+1] int64, sorted_hits [n,2] f32, sorted_ids [n] i32),
    plus sub_off [n_events*n_surf, nb, PHI_SUB] uint16 with ``with_sub``."""
    lib = _load()
    hits = _c(hits, np.float32)
    so = _c(slab_offsets, np.int64)
    nb = lib.or_index_bins(geom.ref)
    n_slabs = n_events * len(geom.wl.surfaces)
    off = np.empty((n_slabs, nb + 1), np.int64)
    sh = np.empty_like(hits)
    si = np.empty(hits.shape[0], np.int32)
    sub = np.empty((n_slabs, nb, PHI_SUB), np.uint16)
    lib.or_build_index(geom.ref, hits.ctypes.data, so.ctypes.data, n_events, off.ctypes.data, sh.ctypes.data,
                       si.ctypes.data, sub.ctypes.data)
    return (off, sh, si, sub) if with_sub else (off, sh, si)


def bin_of(geom: Geometry, surf: int, phi: float, second: float):
    lib = _load()
    a, b = ctypes.c_int(), ctypes.c_int()
    lib.or_bin_of(geom.ref, surf, float(phi), float(second), ctypes.addressof(a), ctypes.addressof(b))
    return a.value, b.value


def search(geom: Geometry, batch, p, C, event: int, surf: int, chi2_cut: float, brute: bool, cap: int = 4096):
    """Hits of (event, surf) with chi2 < cut for predicted state (p, C): (ids, chi2)."""
    lib = _load()
    hits = _c(batch.hits, np.float32)
    hs = _c(batch.hit_surface, np.int32)
    so = _c(batch.slab_offsets, np.int64)
    p = _c(p, np.float64)
    C = _c(C, np.float64)
    ids = np.empty(cap, np.int32)
    c2 = np.empty(cap)
    n = lib.or_search(geom.ref, hits.ctypes.data, hs.ctypes.data, so.ctypes.data, batch.n_events, p.ctypes.data,
                      C.ctypes.data, event, surf, chi2_cut, int(brute), cap, ids.ctypes.data, c2.ctypes.data)
    n = min(n, cap)
    return ids[:n].copy(), c2[:n].copy()


def update(geom: Geometry, p, C, surf: int, hit):
    """Kalman update with one hit (phi, second coordinate): returns (p', C', chi2)."""
    lib = _load()
    p = _c(p, np.float64)
    C = _c(C, np.float64)
    po, Co = np.empty(6), np.empty((6, 6))
    c2 = lib.or_update(geom.ref, p.ctypes.data, C.ctypes.data, surf, float(hit[0]), float(hit[1]), po.ctypes.data,
                       Co.ctypes.data)
    return po, Co, c2


def next_surface(geom: Geometry, p):
    lib = _load()
    p = _c(p, np.float64)
    s = ctypes.c_double()
    k = lib.or_next_surface(geom.ref, p.ctypes.data, ctypes.addressof(s))
    return k, s.value


class OrSteering(ctypes.Structure):
    _fields_ = [("c_barrel", ctypes.c_float), ("c_endcap", ctypes.c_float), ("n", ctypes.c_int * 5),
                ("surf", (ctypes.c_int * 64) * 5)]


def _steering(st):
    """OrSteering from a dict(c_barrel, c_endcap, lists=[5 lists of surface ids]) or None."""
    if st is None:
        return None
    o = OrSteering()
    o.c_barrel, o.c_endcap = float(st["c_barrel"]), float(st["c_endcap"])
    for r, lst in enumerate(st["lists"]):
        o.n[r] = len(lst)
        for q, sid in enumerate(lst):
            o.surf[r][q] = int(sid)
    return o


def find(geom: Geometry, batch, seed_hits, seed_event, *, chi2_cut=None, k_max=None, max_miss=None,
         brute_force: bool = False, n_threads: int = 0, mlp=None, top_n: int = 0, steering=None,
         score_margin: float = 0.0, window: bool = False):
    """Combinatorial finding from seeds; with ``mlp`` = (weights, mean, sd) and top_n > 0 the
    learned proposal keeps the top_n passing hits by score (with ``score_margin`` > 0, of a window
    with two or more passing hits, those of its top_n within the margin of its best score; with
    ``window``, instead, the top_n by score of every hit in the bounding box of the chi2 ellipse go
    on to the chi2 cut when the box holds more than top_n hits, with ``score_margin`` > 0 when it
    holds two or more and only those within the margin of the best); ``steering`` (synth.steering_tables)
    replaces the geometric next-surface rule by the region lists. Returns dict with hits [n,lmax], n_hits, chi2, p, cov,
    status and counters (propagations, passing chi2 evaluations, updates, hits whose chi2 was
    evaluated in a window's bins, hits of the windows limited to the phi sub-bins they touch,
    network evaluations of the learned proposal)."""
    lib = _load()
    wl = geom.wl
    prm = OrFindParams(wl.chi2_cut if chi2_cut is None else chi2_cut, wl.k_max if k_max is None else k_max,
                       wl.max_miss if max_miss is None else max_miss, int(brute_force))
    hits = _c(batch.hits, np.float32)
    hs = _c(batch.hit_surface, np.int32)
    so = _c(batch.slab_offsets, np.int64)
    sh = _c(seed_hits, np.int32)
    se = _c(seed_event, np.int32)
    n = sh.shape[0]
    lmax = wl.lmax
    out = dict(hits=np.empty((n, lmax), np.int32), n_hits=np.empty(n, np.int32), chi2=np.empty(n),
               p=np.empty((n, 6)), cov=np.empty((n, 21)), status=np.empty(n, np.int32))
    counters = np.zeros(6, np.int64)
    lib.or_find(geom.ref, hits.ctypes.data, hs.ctypes.data, so.ctypes.data, batch.n_events, sh.ctypes.data,
                se.ctypes.data, n, lmax, ctypes.byref(prm), n_threads, out["hits"].ctypes.data,
                out["n_hits"].ctypes.data, out["chi2"].ctypes.data, out["p"].ctypes.data, out["cov"].ctypes.data,
                out["status"].ctypes.data, counters.ctypes.data, *_mlp_ptrs(mlp), int(top_n),
                None if steering is None else ctypes.byref(_steering(steering)), float(score_margin), int(bool(window)))
    out["counters"] = counters
    return out


MLP_NPARAMS = 14 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def _mlp_ptrs(mlp):
    if mlp is None:
        return None, None, None
    w, mean, sd = (np.ascontiguousarray(a, np.float64) for a in mlp)
    _mlp_ptrs.keep = (w, mean, sd)  # alive for the duration of the call
    return w.ctypes.data, mean.ctypes.data, sd.ctypes.data


def find_pairs(geom: Geometry, batch, seed_hits, seed_event, seed_track, *, cap: int = 10_000_000,
               n_threads: int = 0):
    """Training pairs of the learned proposal: every passing (candidate, hit) pair of the plain
    finding from these seeds. Returns (features [n,14] float32, labels [n] float32)."""
    lib = _load()
    wl = geom.wl
    prm = OrFindParams(wl.chi2_cut, wl.k_max, wl.max_miss, 0)
    sh = _c(seed_hits, np.int32)
    se = _c(seed_event, np.int32)
    stk = _c(seed_track, np.int32)
    feats = np.empty((cap, 14), np.float32)
    labels = np.empty(cap, np.float32)
    n = lib.or_find_pairs(geom.ref, _c(batch.hits, np.float32).ctypes.data, _c(batch.hit_surface, np.int32).ctypes.data,
                          _c(batch.slab_offsets, np.int64).ctypes.data, batch.n_events, sh.ctypes.data, se.ctypes.data,
                          stk.ctypes.data, _c(batch.hit_sim, np.int32).ctypes.data, sh.shape[0], wl.lmax,
                          ctypes.byref(prm), n_threads, cap, feats.ctypes.data, labels.ctypes.data)
    n = min(n, cap)
    return feats[:n].copy(), labels[:n].copy()


def pair_features(geom: Geometry, surf: int, p, C, hit):
    """The learned proposal's 14 features of a predicted state (p, C) and a hit (phi, v)."""
    lib = _load()
    p = _c(p, np.float64)
    C = _c(C, np.float64)
    f = np.empty(14)
    lib.or_pair_features(geom.ref, int(surf), p.ctypes.data, C.ctypes.data, float(hit[0]), float(hit[1]), f.ctypes.data)
    return f


def mlp_forward(w, xs):
    """Logits of the MLP for standardised features xs [n,14] (FP64)."""
    lib = _load()
    w = _c(w, np.float64)
    xs = _c(xs, np.float64)
    out = np.empty(xs.shape[0])
    lib.or_mlp_forward(w.ctypes.data, xs.ctypes.data, xs.shape[0], out.ctypes.data)
    return out


def mlp_loss_grad(w, xs, y):
    """Mean BCE-with-logits loss over the batch and its gradient (FP64)."""
    lib = _load()
    w = _c(w, np.float64)
    xs = _c(xs, np.float64)
    y = _c(y, np.float64)
    g = np.empty(MLP_NPARAMS)
    loss = lib.or_mlp_loss_grad(w.ctypes.data, xs.ctypes.data, y.ctypes.data, xs.shape[0], g.ctypes.data)
    return loss, g


def adam(w, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place on (w, m, v) (FP64 arrays)."""
    lib = _load()
    for a in (w, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib.or_adam(w.ctypes.data, grad.ctypes.data, m.ctypes.data, v.ctypes.data, int(t), lr, b1, b2, eps)


def unpack_cov(c21):
    """Packed upper triangle (row-major, i <= j) -> full symmetric [..., 6, 6]."""
    c21 = np.asarray(c21)
    out = np.empty(c21.shape[:-1] + (6, 6), c21.dtype)
    k = 0
    for i in range(6):
        for j in range(i, 6):
            out[..., i, j] = c21[..., k]
            out[..., j, i] = c21[..., k]
            k += 1
    return out


def seed_params(geom: Geometry, batch, seed_hits):
    """(kappa, phi, theta) of each seed from its three hits ([n, 3]; NaN when no seed)."""
    lib = _load()
    sh = _c(seed_hits, np.int32)
    out = np.empty((sh.shape[0], 3))
    lib.or_seed_params(geom.ref, _c(batch.hits, np.float32).ctypes.data, _c(batch.hit_surface, np.int32).ctypes.data,
                       sh.ctypes.data, sh.shape[0], out.ctypes.data)
    return out


def clean_seeds(seed_hits, seed_event, params, dphi: float = 0.02, dtheta: float = 0.05):
    """Seed cleaning: keep[n] (0 for a seed with a lower-index duplicate)."""
    lib = _load()
    sh, se, pr = _c(seed_hits, np.int32), _c(seed_event, np.int32), _c(params, np.float64)
    keep = np.empty(sh.shape[0], np.int32)
    lib.or_clean_seeds(sh.ctypes.data, se.ctypes.data, pr.ctypes.data, sh.shape[0], float(dphi), float(dtheta),
                       keep.ctypes.data)
    return keep


def remove_duplicates(hits, n_hits, chi2, phi, theta, track_event, dphi: float = 0.02, dtheta: float = 0.05):
    """Duplicate-track removal: keep[n] (0 for a track with a better duplicate)."""
    lib = _load()
    h = _c(hits, np.int32)
    keep = np.empty(h.shape[0], np.int32)
    lib.or_remove_duplicates(h.ctypes.data, _c(n_hits, np.int32).ctypes.data, _c(chi2, np.float64).ctypes.data,
                             _c(phi, np.float64).ctypes.data, _c(theta, np.float64).ctypes.data,
                             _c(track_event, np.int32).ctypes.data, h.shape[0], h.shape[1], float(dphi),
                             float(dtheta), keep.ctypes.data)
    return keep


def majority_sim(batch, found_hits, found_nhits, min_hits: int = 10, match_frac: float = 0.5):
    """Simulated track each found track is matched to, whatever its seed (-1: none): the sim track
    holding more than ``match_frac`` of the track's hits, for tracks with >= min(min_hits, that
    sim track's crossings - 1) hits (the paper's hit-fraction matching, Sec. 4)."""
    fh = np.asarray(found_hits)
    nh = np.asarray(found_nhits)
    out = np.full(len(fh), -1, np.int64)
    for i in range(len(fh)):
        sims = batch.hit_sim[fh[i][fh[i] >= 0]]
        sims = sims[sims >= 0]
        if len(sims) == 0:
            continue
        vals, cnt = np.unique(sims, return_counts=True)
        t = int(vals[np.argmax(cnt)])
        if cnt.max() > match_frac * (fh[i] >= 0).sum() and nh[i] >= min(min_hits, int(batch.track_nhits[t]) - 1):
            out[i] = t
    return out


def track_rates(batch, seed_track, matched, keep=None, min_hits: int = 10, track_sim=None):
    """Per simulated track (several seeds may share one): efficiency = reference tracks (>=
    min_hits hits, with a seed) with at least one matched kept track; duplicate rate = reference
    tracks with two or more (the paper's duplicate track rate, Sec. 4). A track counts for its
    seed's sim track, or, with ``track_sim`` (majority_sim), for the sim track it is matched to."""
    st = np.asarray(seed_track)
    m = np.asarray(matched, bool) & (np.ones(len(st), bool) if keep is None else np.asarray(keep) != 0)
    owner = st
    if track_sim is not None:
        owner = np.asarray(track_sim)
        m &= owner >= 0
    counts = np.bincount(owner[m], minlength=batch.n_tracks)
    ref = np.zeros(batch.n_tracks, bool)
    ref[st] = True
    ref &= batch.track_nhits >= min_hits
    return float((counts[ref] >= 1).mean()), float((counts[ref] >= 2).mean())


def efficiency(batch, seed_track, found_hits, found_nhits, min_hits: int = 10, match_frac: float = 0.5):
    """Efficiency and fake rate, adapted from the paper's standalone validation (Sec. 4): a
    reference track is a sim track with >= ``min_hits`` hits; a seed's best track is matched to the
    seed's sim track when it has >= min(min_hits, crossings - 1) hits and at least ``match_frac``
    of its hits beyond the 3 seed hits belong to that sim track (the paper uses 4-hit seeds and
    the same 50% rule). Efficiency = matched reference tracks / reference tracks; fake rate =
    unmatched best tracks / all best tracks. Returns (efficiency, fake_rate, matched[n_seeds])."""
    seed_track = np.asarray(seed_track)
    fh = np.asarray(found_hits)
    nh = np.asarray(found_nhits)
    n_true = batch.track_nhits[seed_track]
    matched = np.zeros(len(seed_track), bool)
    for i in range(len(seed_track)):
        need = min(min_hits, int(n_true[i]) - 1)
        if nh[i] < need:
            continue
        ext = [h for h in fh[i, 3:] if h >= 0]
        if not ext:
            continue
        own = sum(1 for h in ext if batch.hit_sim[h] == seed_track[i])
        matched[i] = own >= match_frac * len(ext)
    ref = n_true >= min_hits
    eff = matched[ref].mean() if ref.any() else float("nan")
    fake = 1.0 - matched.mean() if len(matched) else float("nan")
    return float(eff), float(fake), matched
