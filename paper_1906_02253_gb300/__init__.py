"""kfgb: Kalman-filter track fitting and combinatorial track finding on GB300 (sm_103a).

Thin binding over the C ABI in ``include/kfgb.h`` (``_build/libkfgb.so``): each function takes
PyTorch CUDA tensors, passes their device pointers and the current stream, and returns the
output tensors. No arithmetic happens here and there is no fallback: if the CUDA library is not
built or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libkfgb.so")
_lib = None
_lock = threading.Lock()

KF_OK, KF_ERR_ARG, KF_ERR_CAPACITY, KF_ERR_CUDA, KF_ERR_TIMEOUT = 0, -1, -2, -3, -4
KF_BARREL, KF_DISK = 0, 1
KF_MAX_SURF, KF_MAX_LMAX, KF_MAX_K, KF_MAX_SLAB_HITS = 64, 31, 16, 32768


class KfError(RuntimeError):
    pass


class KfSurface(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("r_or_z", ctypes.c_float), ("lo", ctypes.c_float), ("hi", ctypes.c_float),
                ("x_over_x0", ctypes.c_float), ("n_phi", ctypes.c_int), ("n_2nd", ctypes.c_int)]


class KfGeometry(ctypes.Structure):
    _fields_ = [("bz", ctypes.c_float), ("n_surf", ctypes.c_int), ("surf", ctypes.POINTER(KfSurface)),
                ("sigma_rphi", ctypes.c_float), ("sigma_2nd", ctypes.c_float), ("prior", ctypes.c_float * 5),
                ("ms_off", ctypes.c_int), ("material", ctypes.c_void_p), ("eloss", ctypes.c_float),
                ("mass", ctypes.c_float), ("field_z2", ctypes.c_float), ("field_r2", ctypes.c_float)]


MAT_NODES = 8  # KF_MAT_NODES


class KfHitIndex(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int), ("n_bins", ctypes.c_int), ("bin_off", ctypes.c_void_p),
                ("sorted_hits", ctypes.c_void_p), ("sorted_ids", ctypes.c_void_p), ("sorted_rec", ctypes.c_void_p), ("sub_off", ctypes.c_void_p)]


N_REGIONS, MAX_SURF = 5, 64  # KF_N_REGIONS, KF_MAX_SURF


class KfSteering(ctypes.Structure):
    _fields_ = [("c_barrel", ctypes.c_float), ("c_endcap", ctypes.c_float), ("n", ctypes.c_int * N_REGIONS),
                ("surf", (ctypes.c_byte * MAX_SURF) * N_REGIONS)]


class KfFindParams(ctypes.Structure):
    _fields_ = [("chi2_cut", ctypes.c_float), ("k_max", ctypes.c_int), ("max_miss", ctypes.c_int),
                ("lmax", ctypes.c_int), ("block_threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("mlp", ctypes.c_void_p), ("top_n", ctypes.c_int), ("k_capacity", ctypes.c_int),
                ("steering", ctypes.POINTER(KfSteering)), ("seed_keep", ctypes.c_void_p),
                ("score_margin", ctypes.c_float), ("adaptive_capacity", ctypes.c_int), ("window_ranking", ctypes.c_int)]


EXPORTS = ("kf_build_hit_index", "kf_index_bins", "kf_fit_tracks", "kf_find_workspace_size", "kf_find_tracks",
           "kf_find_tracks_static", "kf_mlp_forward", "kf_mlp_loss_grad", "kf_mlp_adam", "kf_autotune_find",
           "kf_autotune_fit", "kf_status_string", "kf_dedup_workspace_size", "kf_clean_seeds",
           "kf_remove_duplicates", "kf_fp32_fma_probe", "kf_math_probe", "kf_seed_states",
           "kf_wait_probe", "kf_mlp_finder_scores")
MLP_PARAMS, MLP_BUFFER = 5185, 5213
KF_MLP_FRAG_BYTES = 20480  # the finder's tensor-core operands of the network (kfgb.h)
PHI_SUB = 8  # KF_PHI_SUB: phi sub-bins per phi bin of the hit index


def load_library(path: str = LIB_PATH):
    """Load ``libkfgb.so`` (raises if it is missing: there is no CPU path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise KfError(f"{path} is not built; run __graft_entry__.build() (nvcc, sm_103a)")
            lib = ctypes.CDLL(path)
            P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            G = ctypes.POINTER(KfGeometry)
            lib.kf_build_hit_index.restype = I
            lib.kf_build_hit_index.argtypes = [G, P, P, I, I, ctypes.POINTER(KfHitIndex), P, P]
            lib.kf_index_bins.restype = I
            lib.kf_index_bins.argtypes = [G]
            lib.kf_fit_tracks.restype = I
            lib.kf_fit_tracks.argtypes = [G, P, P, P, I, I, P, P, P, P, P, I, P]
            lib.kf_find_workspace_size.restype = S
            lib.kf_find_workspace_size.argtypes = [I, ctypes.POINTER(KfFindParams)]
            lib.kf_find_tracks.restype = I
            lib.kf_find_tracks.argtypes = [G, ctypes.POINTER(KfHitIndex), P, P, P, P, I, ctypes.POINTER(KfFindParams),
                                           P, P, P, P, P, P, P, S, P]
            lib.kf_mlp_forward.restype = I
            lib.kf_mlp_forward.argtypes = [P, P, I, P, P]
            lib.kf_mlp_finder_scores.restype = I
            lib.kf_mlp_finder_scores.argtypes = [P, P, I, P, P, P]
            lib.kf_mlp_loss_grad.restype = I
            lib.kf_mlp_loss_grad.argtypes = [P, P, P, I, P, P, P]
            lib.kf_mlp_adam.restype = I
            lib.kf_mlp_adam.argtypes = [P, P, P, P, I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, P]
            lib.kf_autotune_find.restype = I
            lib.kf_autotune_find.argtypes = [G, ctypes.POINTER(KfHitIndex), P, P, P, P, I,
                                             ctypes.POINTER(KfFindParams), P, P, P, P, P, P, P, S,
                                             ctypes.POINTER(ctypes.c_float), P]
            lib.kf_autotune_fit.restype = I
            lib.kf_autotune_fit.argtypes = [G, P, P, P, I, I, P, P, P, P, P, ctypes.POINTER(ctypes.c_int),
                                            ctypes.POINTER(ctypes.c_float), P]
            lib.kf_dedup_workspace_size.restype = S
            lib.kf_dedup_workspace_size.argtypes = [I, I, I]
            lib.kf_clean_seeds.restype = I
            lib.kf_clean_seeds.argtypes = [G, P, P, I, P, P, I, ctypes.c_float, ctypes.c_float, P, P, S, P]
            lib.kf_remove_duplicates.restype = I
            lib.kf_remove_duplicates.argtypes = [P, P, P, P, P, I, I, I, ctypes.c_float, ctypes.c_float, P, P, S, P]
            lib.kf_fp32_fma_probe.restype = I
            lib.kf_fp32_fma_probe.argtypes = [P, I, I, ctypes.POINTER(ctypes.c_longlong), P]
            lib.kf_seed_states.restype = I
            lib.kf_seed_states.argtypes = [G, P, P, P, P, I, I, P, P, P]
            lib.kf_math_probe.restype = I
            lib.kf_math_probe.argtypes = [I, P, P, I, P, P, P, P]
            lib.kf_wait_probe.restype = I
            lib.kf_wait_probe.argtypes = [I, P, P]
            lib.kf_status_string.restype = ctypes.c_char_p
            lib.kf_status_string.argtypes = [I]
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != KF_OK:
        msg = load_library().kf_status_string(rc).decode()
        raise KfError(f"{what} failed: {msg} ({rc})")


class Geometry:
    """C-ABI geometry built from any object with ``surfaces`` (type, r_or_z, lo, hi, x_over_x0,
    n_phi, n_2nd), ``bz``, ``sigma_rphi``, ``sigma_2nd``, ``prior``, ``ms_on`` and optionally
    ``material`` ([n_surf][MAT_NODES] x/X0), ``eloss``, ``mass``, ``field_z2`` and ``field_r2``."""

    def __init__(self, wl):
        self.wl = wl
        n = len(wl.surfaces)
        self._surf = (KfSurface * n)()
        ms = getattr(wl, "ms_on", True)
        for i, s in enumerate(wl.surfaces):
            self._surf[i] = KfSurface(s.type, s.r_or_z, s.lo, s.hi, s.x_over_x0, s.n_phi, s.n_2nd)
        mat = getattr(wl, "material", None)
        self._mat = None if mat is None else np.ascontiguousarray(mat, dtype=np.float32)
        if self._mat is not None and self._mat.shape != (n, MAT_NODES):
            raise KfError(f"material map must be [{n}][{MAT_NODES}]")
        self.g = KfGeometry(wl.bz, n, ctypes.cast(self._surf, ctypes.POINTER(KfSurface)), wl.sigma_rphi, wl.sigma_2nd,
                            (ctypes.c_float * 5)(*wl.prior), int(not ms),
                            None if self._mat is None else self._mat.ctypes.data, getattr(wl, "eloss", 0.0),
                            getattr(wl, "mass", 0.13957), getattr(wl, "field_z2", 0.0),
                            getattr(wl, "field_r2", 0.0))
        self.n_surf = n
        self.n_bins = load_library().kf_index_bins(ctypes.byref(self.g))
        if self.n_bins < 0:
            _check(self.n_bins, "geometry")

    @property
    def ref(self):
        return ctypes.byref(self.g)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _cuda(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise KfError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise KfError(f"{name} must be {dtype}")
    if not t.is_contiguous():
        raise KfError(f"{name} must be contiguous")
    return t


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class HitIndex:
    """Device buffers of a hit index (caller-owned tensors)."""

    def __init__(self, geom: Geometry, n_events: int, n_hits: int, device="cuda"):
        self.n_events = n_events
        self.n_bins = geom.n_bins
        self.bin_off = torch.empty((n_events * geom.n_surf, geom.n_bins + 1), dtype=torch.int32, device=device)
        self.sorted_hits = torch.empty((n_hits, 2), dtype=torch.float32, device=device)
        self.sorted_ids = torch.empty(n_hits, dtype=torch.int32, device=device)
        self.sorted_rec = torch.empty((n_hits, 4), dtype=torch.float32, device=device)
        # uint16 sub-bin offsets, held as int16 (torch has no uint16 on every supported version)
        self.sub_off = torch.empty((n_events * geom.n_surf, geom.n_bins, PHI_SUB), dtype=torch.int16, device=device)
        self.c = KfHitIndex(n_events, self.n_bins, self.bin_off.data_ptr(), self.sorted_hits.data_ptr(),
                            self.sorted_ids.data_ptr(), self.sorted_rec.data_ptr(), self.sub_off.data_ptr())


def build_hit_index(geom: Geometry, hits, slab_offsets, n_events: int, max_slab_hits: int, index: HitIndex = None,
                    status=None, stream=None) -> HitIndex:
    """kf_build_hit_index: hits [n,2] f32, slab_offsets [n_events*n_surf+1] i32 (device)."""
    lib = load_library()
    _cuda(hits, torch.float32, "hits")
    _cuda(slab_offsets, torch.int32, "slab_offsets")
    if index is None:
        index = HitIndex(geom, n_events, hits.shape[0], hits.device)
    rc = lib.kf_build_hit_index(geom.ref, _ptr(hits), _ptr(slab_offsets), n_events, int(max_slab_hits),
                                ctypes.byref(index.c), _ptr(status), _stream(stream))
    _check(rc, "kf_build_hit_index")
    return index


def fit_tracks(geom: Geometry, hits, hit_surface, track_hits, out: dict = None, block_threads: int = 0,
               stream=None) -> dict:
    """kf_fit_tracks: track_hits [lmax, n] i32 (structure of arrays). Returns state [6,n],
    cov [21,n], chi2 [n], ndof [n], status [n]."""
    lib = load_library()
    _cuda(hits, torch.float32, "hits")
    _cuda(hit_surface, torch.int32, "hit_surface")
    _cuda(track_hits, torch.int32, "track_hits")
    lmax, n = track_hits.shape
    dev = hits.device
    if out is None:
        out = dict(state=torch.empty((6, n), dtype=torch.float32, device=dev),
                   cov=torch.empty((21, n), dtype=torch.float32, device=dev),
                   chi2=torch.empty(n, dtype=torch.float32, device=dev),
                   ndof=torch.empty(n, dtype=torch.int32, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev))
    rc = lib.kf_fit_tracks(geom.ref, _ptr(hits), _ptr(hit_surface), _ptr(track_hits), n, lmax, _ptr(out["state"]),
                           _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out["ndof"]), _ptr(out["status"]),
                           int(block_threads), _stream(stream))
    _check(rc, "kf_fit_tracks")
    return out


def steering(tables: dict) -> KfSteering:
    """KfSteering from dict(c_barrel, c_endcap, lists=[5 lists of surface ids]) (marshalling only)."""
    st = KfSteering()
    st.c_barrel, st.c_endcap = float(tables["c_barrel"]), float(tables["c_endcap"])
    lists = tables["lists"]
    if len(lists) != N_REGIONS:
        raise KfError(f"steering needs {N_REGIONS} region lists")
    for r, lst in enumerate(lists):
        if len(lst) > MAX_SURF:
            raise KfError("steering list longer than the surface limit")
        st.n[r] = len(lst)
        for q, sid in enumerate(lst):
            st.surf[r][q] = int(sid)
    return st


def find_params(chi2_cut: float, k_max: int, max_miss: int, lmax: int, block_threads: int = 0,
                blocks_per_sm: int = 0, mlp=None, top_n: int = 0, k_capacity: int = 0,
                steering_tables: dict = None, seed_keep=None, score_margin: float = 0.0,
                adaptive_capacity: int = 0, window_ranking: bool = False) -> KfFindParams:
    """Finder settings; ``mlp`` is a device tensor of MLP_BUFFER floats (learned proposal);
    ``steering_tables`` (dict of region lists) selects region steering instead of the geometric
    next-surface rule; ``score_margin`` > 0 switches the learned proposal to its score-margin rule;
    ``adaptive_capacity`` > 0 runs the finder in two passes; ``window_ranking`` ranks the learned
    proposal's whole window before the chi2 cut (see kfgb.h)."""
    if mlp is not None:
        _cuda(mlp, torch.float32, "mlp")
        if mlp.numel() != MLP_BUFFER:
            raise KfError(f"mlp must hold {MLP_BUFFER} floats")
    st = None if steering_tables is None else steering(steering_tables)
    if seed_keep is not None:
        _cuda(seed_keep, torch.int32, "seed_keep")
    prm = KfFindParams(chi2_cut, k_max, max_miss, lmax, block_threads, blocks_per_sm,
                       None if mlp is None else mlp.data_ptr(), int(top_n), int(k_capacity),
                       None if st is None else ctypes.pointer(st), None if seed_keep is None else seed_keep.data_ptr(),
                       float(score_margin), int(adaptive_capacity), int(bool(window_ranking)))
    prm._mlp_ref = mlp  # keep the buffers alive with the parameters
    prm._steer_ref = st
    prm._keep_ref = seed_keep
    return prm


def dedup_workspace_size(n_items: int, refs_per_item: int, n_hits: int) -> int:
    """kf_dedup_workspace_size: bytes for kf_clean_seeds (refs 3) or kf_remove_duplicates (lmax)."""
    return int(load_library().kf_dedup_workspace_size(n_items, refs_per_item, n_hits))


def clean_seeds(geom: Geometry, hits, hit_surface, seed_hits, seed_event, dphi: float = 0.02, dtheta: float = 0.05,
                keep=None, workspace=None, stream=None):
    """kf_clean_seeds: keep [n_seeds] int32 (0: a seed with a lower-index duplicate)."""
    lib = load_library()
    for t, nm in ((hit_surface, "hit_surface"), (seed_hits, "seed_hits"), (seed_event, "seed_event")):
        _cuda(t, torch.int32, nm)
    _cuda(hits, torch.float32, "hits")
    n, nh = seed_hits.shape[1], hits.shape[0]
    if keep is None:
        keep = torch.empty(n, dtype=torch.int32, device=hits.device)
    ws = workspace
    if ws is None:
        ws = torch.empty(max(int(lib.kf_dedup_workspace_size(n, 3, nh)), 256), dtype=torch.uint8, device=hits.device)
    rc = lib.kf_clean_seeds(geom.ref, _ptr(hits), _ptr(hit_surface), nh, _ptr(seed_hits), _ptr(seed_event), n,
                            float(dphi), float(dtheta), _ptr(keep), _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "kf_clean_seeds")
    return keep


def remove_duplicates(track_hits, nhits, chi2, state, track_event, n_hits: int, dphi: float = 0.02,
                      dtheta: float = 0.05, keep=None, workspace=None, stream=None):
    """kf_remove_duplicates on the finder's outputs: keep [n_tracks] int32 (0: a duplicate)."""
    lib = load_library()
    for t, nm in ((track_hits, "track_hits"), (nhits, "nhits"), (track_event, "track_event")):
        _cuda(t, torch.int32, nm)
    _cuda(chi2, torch.float32, "chi2")
    _cuda(state, torch.float32, "state")
    lmax, n = track_hits.shape
    if keep is None:
        keep = torch.empty(n, dtype=torch.int32, device=track_hits.device)
    ws = workspace
    if ws is None:
        ws = torch.empty(max(int(lib.kf_dedup_workspace_size(n, lmax, n_hits)), 256), dtype=torch.uint8,
                         device=track_hits.device)
    rc = lib.kf_remove_duplicates(_ptr(track_hits), _ptr(nhits), _ptr(chi2), _ptr(state), _ptr(track_event), n, lmax,
                                  int(n_hits), float(dphi), float(dtheta), _ptr(keep), _ptr(ws), ws.numel(),
                                  _stream(stream))
    _check(rc, "kf_remove_duplicates")
    return keep


def fp32_fma_rate(blocks: int = 0, iters: int = 4096, reps: int = 3, stream=None) -> float:
    """kf_fp32_fma_probe timed with CUDA events: the best of `reps` launches, TFLOP/s (FMA = 2)."""
    lib = load_library()
    dev = torch.cuda.current_device()
    if blocks <= 0:
        blocks = 8 * torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(blocks, dtype=torch.float32, device="cuda")
    s = stream if stream is not None else torch.cuda.current_stream()
    flops = ctypes.c_longlong()
    best = 0.0
    for _ in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        _check(lib.kf_fp32_fma_probe(_ptr(sink), blocks, iters, ctypes.byref(flops), _stream(s)), "kf_fp32_fma_probe")
        b.record(s)
        b.synchronize()
        best = max(best, flops.value / (a.elapsed_time(b) / 1000.0) / 1e12)
    return best


PROBE_SINCOS, PROBE_ATAN_SMALL, PROBE_HALF_ANGLE = 0, 1, 2  # KF_PROBE_*


def wait_probe(limit_us: int, stream=None):
    """kf_wait_probe: the tensor-core kernels' bounded mbarrier wait, once with no arrival (gives up
    after limit_us) and once after the arrival. Returns (first completed, second completed, first
    wait's ns) as an int64 CUDA tensor."""
    out = torch.full((3,), -1, dtype=torch.int64, device="cuda")
    _check(load_library().kf_wait_probe(int(limit_us), _ptr(out), _stream(stream)), "kf_wait_probe")
    return out


def math_probe(fn: int, a, b=None, stream=None):
    """kf_math_probe: the path's hand-written trigonometry on FP32 CUDA tensors a (and b for the
    small-angle arctangent). Returns three tensors (o0, o1, o2) of a's shape."""
    lib = load_library()
    a = _cuda(a, torch.float32, "a").contiguous()
    b = None if b is None else _cuda(b, torch.float32, "b").contiguous()
    o = [torch.empty_like(a) for _ in range(3)]
    _check(lib.kf_math_probe(int(fn), _ptr(a), _ptr(b), a.numel(), _ptr(o[0]), _ptr(o[1]), _ptr(o[2]), _stream(stream)),
           "kf_math_probe")
    return tuple(o)


def seed_states(geom: Geometry, hits, hit_surface, seed_hits, seed_event, n_events: int, out=None, stream=None):
    """kf_seed_states: the fitted state of every seed at its third hit. Returns (state [28, n]
    float32: p[6], packed C[21], chi2 (-1: failed seed), surface [n] int32 of hit 3)."""
    for t, nm in ((hit_surface, "hit_surface"), (seed_hits, "seed_hits"), (seed_event, "seed_event")):
        _cuda(t, torch.int32, nm)
    _cuda(hits, torch.float32, "hits")
    n = seed_hits.shape[1]
    if out is None:
        out = (torch.empty((28, n), dtype=torch.float32, device=hits.device),
               torch.empty(n, dtype=torch.int32, device=hits.device))
    _check(load_library().kf_seed_states(geom.ref, _ptr(hits), _ptr(hit_surface), _ptr(seed_hits), _ptr(seed_event),
                                         n, int(n_events), _ptr(out[0]), _ptr(out[1]), _stream(stream)),
           "kf_seed_states")
    return out


def find_workspace_size(n_seeds: int, params: KfFindParams) -> int:
    return int(load_library().kf_find_workspace_size(n_seeds, ctypes.byref(params)))


def find_tracks(geom: Geometry, index: HitIndex, hits, hit_surface, seed_hits, seed_event, params: KfFindParams,
                out: dict = None, workspace=None, stream=None) -> dict:
    """kf_find_tracks: seed_hits [3, n] i32 (structure of arrays), seed_event [n] i32. Returns
    hits [lmax, n], nhits, chi2, state [6,n], cov [21,n], status."""
    lib = load_library()
    _cuda(hits, torch.float32, "hits")
    _cuda(hit_surface, torch.int32, "hit_surface")
    _cuda(seed_hits, torch.int32, "seed_hits")
    _cuda(seed_event, torch.int32, "seed_event")
    n = seed_hits.shape[1]
    dev = hits.device
    lmax = params.lmax
    if out is None:
        out = dict(hits=torch.empty((lmax, n), dtype=torch.int32, device=dev),
                   nhits=torch.empty(n, dtype=torch.int32, device=dev),
                   chi2=torch.empty(n, dtype=torch.float32, device=dev),
                   state=torch.empty((6, n), dtype=torch.float32, device=dev),
                   cov=torch.empty((21, n), dtype=torch.float32, device=dev),
                   status=torch.empty(n, dtype=torch.int32, device=dev))
    ws_bytes = find_workspace_size(n, params)
    if ws_bytes == 0 and n > 0:
        raise KfError("kf_find_workspace_size rejected the parameters")
    if workspace is None or workspace.numel() < ws_bytes:
        workspace = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device=dev)
    rc = lib.kf_find_tracks(geom.ref, ctypes.byref(index.c), _ptr(hits), _ptr(hit_surface), _ptr(seed_hits),
                            _ptr(seed_event), n, ctypes.byref(params), _ptr(out["hits"]), _ptr(out["nhits"]),
                            _ptr(out["chi2"]), _ptr(out["state"]), _ptr(out["cov"]), _ptr(out["status"]),
                            _ptr(workspace), workspace.numel(), _stream(stream))
    _check(rc, "kf_find_tracks")
    out["workspace"] = workspace
    return out


def to_device_event_batch(batch, device="cuda") -> dict:
    """Move a generated event batch's inputs to the device in the layouts the ABI takes."""
    seeds, st = batch.seeds()
    return dict(
        hits=torch.from_numpy(np.ascontiguousarray(batch.hits)).to(device),
        hit_surface=torch.from_numpy(np.ascontiguousarray(batch.hit_surface)).to(device),
        slab_offsets=torch.from_numpy(batch.slab_offsets.astype(np.int32)).to(device),
        track_hits=torch.from_numpy(np.ascontiguousarray(batch.track_hits.T)).to(device),
        seed_hits=torch.from_numpy(np.ascontiguousarray(seeds.T)).to(device),
        seed_event=torch.from_numpy(batch.track_event[st].astype(np.int32)).to(device),
        seed_track=st,
        max_slab_hits=int(np.diff(batch.slab_offsets).max()) if batch.slab_offsets.size > 1 else 0,
    )


# ------------------------------------------------------------------------------------------------
# Learned hit proposal: network buffer, inference and training through the C ABI
# ------------------------------------------------------------------------------------------------

def mlp_buffer(weights, mean, sd, device="cuda"):
    """Device parameter buffer: KF_MLP_PARAMS weights, then the feature mean[14] and sd[14]."""
    buf = np.concatenate([np.asarray(weights, np.float32).ravel(), np.asarray(mean, np.float32).ravel(),
                          np.asarray(sd, np.float32).ravel()])
    if buf.size != MLP_BUFFER:
        raise KfError(f"expected {MLP_BUFFER} values, got {buf.size}")
    return torch.from_numpy(buf).to(device)


def mlp_forward(params, features, out=None, stream=None):
    """Logits of raw feature rows [n, 14] (kf_mlp_forward)."""
    _cuda(params, torch.float32, "params")
    _cuda(features, torch.float32, "features")
    n = features.shape[0]
    out = torch.empty(n, dtype=torch.float32, device=features.device) if out is None else out
    _check(load_library().kf_mlp_forward(_ptr(params), _ptr(features), n, _ptr(out), _stream(stream)), "kf_mlp_forward")
    return out


def mlp_finder_scores(params, features, out=None, stream=None):
    """Logits of raw feature rows [n, 14] evaluated as the finder scores its pairs
    (kf_mlp_finder_scores: warp-level tensor-core MMAs with the fp16 two-part split)."""
    _cuda(params, torch.float32, "params")
    features = _cuda(features, torch.float32, "features").contiguous()
    n = features.shape[0]
    out = torch.empty(n, dtype=torch.float32, device=features.device) if out is None else out
    ws = torch.empty(KF_MLP_FRAG_BYTES, dtype=torch.uint8, device=features.device)
    _check(load_library().kf_mlp_finder_scores(_ptr(params), _ptr(features), n, _ptr(out), _ptr(ws), _stream(stream)),
           "kf_mlp_finder_scores")
    return out


def mlp_loss_grad(params, features, labels, grad=None, loss=None, stream=None):
    """Mean BCE-with-logits loss and its gradient over the weights (kf_mlp_loss_grad)."""
    _cuda(params, torch.float32, "params")
    _cuda(features, torch.float32, "features")
    _cuda(labels, torch.float32, "labels")
    dev = params.device
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=dev) if grad is None else grad
    loss = torch.empty(1, dtype=torch.float32, device=dev) if loss is None else loss
    _check(load_library().kf_mlp_loss_grad(_ptr(params), _ptr(features), _ptr(labels), features.shape[0], _ptr(grad),
                                           _ptr(loss), _stream(stream)), "kf_mlp_loss_grad")
    return loss, grad


def mlp_adam(params, grad, m, v, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8, stream=None):
    """One Adam step on the weights in params (kf_mlp_adam)."""
    _check(load_library().kf_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), lr, beta1, beta2, eps,
                                      _stream(stream)), "kf_mlp_adam")


def mlp_train(params, features, labels, epochs: int = 3, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
              log=None, lr_halving: int = 0):
    """Train the network in params on (features, labels) with minibatch Adam, all arithmetic in the
    library's kernels (forward, backward, Adam); the host only picks the minibatches. With
    lr_halving > 0 the learning rate halves every lr_halving epochs."""
    dev = params.device
    n = features.shape[0]
    m = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
    v = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=dev)
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    step = 0
    history = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(dev)
        fx, fy = features[perm].contiguous(), labels[perm].contiguous()
        lr_ep = lr * (0.5 ** (ep // lr_halving) if lr_halving > 0 else 1.0)
        for b0 in range(0, n - batch + 1, batch):
            step += 1
            mlp_loss_grad(params, fx[b0:b0 + batch], fy[b0:b0 + batch], grad, loss)
            mlp_adam(params, grad, m, v, step, lr_ep)
        full, _ = mlp_loss_grad(params, features, labels, grad, loss)
        history.append(float(full.item()))
        if log:
            log(f"epoch {ep}: loss {history[-1]:.4f}")
    return history


# ------------------------------------------------------------------------------------------------
# Autotuning (kf_autotune_find / kf_autotune_fit) and its cache
# ------------------------------------------------------------------------------------------------

def autotune_find(geom: Geometry, index: HitIndex, hits, hit_surface, seed_hits, seed_event, params: KfFindParams,
                  stream=None):
    """Time every block size, candidate capacity and (k_max > 4) adaptive capacity on these seeds (a
    calibration subset) and return (tuned params, best ms). Synchronises the stream."""
    # Workspace for the largest configuration tried: adaptive capacity adds its overflow list.
    wide = KfFindParams.from_buffer_copy(params)
    if params.k_max > 4 and (not (params.mlp and params.top_n > 0) or params.top_n <= 4):
        wide.adaptive_capacity = 4  # the overflow list is as long for every first-pass capacity
    n = seed_hits.shape[1]
    ws = torch.empty(max(find_workspace_size(n, wide), find_workspace_size(n, params), 256), dtype=torch.uint8,
                     device=seed_hits.device)
    out = find_tracks(geom, index, hits, hit_surface, seed_hits, seed_event, params, workspace=ws, stream=stream)
    tuned = KfFindParams.from_buffer_copy(params)
    tuned._mlp_ref = getattr(params, "_mlp_ref", None)  # keep what the copied pointers point to alive
    tuned._steer_ref = getattr(params, "_steer_ref", None)
    tuned._keep_ref = getattr(params, "_keep_ref", None)
    ms = ctypes.c_float()
    rc = load_library().kf_autotune_find(geom.ref, ctypes.byref(index.c), _ptr(hits), _ptr(hit_surface),
                                         _ptr(seed_hits), _ptr(seed_event), seed_hits.shape[1], ctypes.byref(tuned),
                                         _ptr(out["hits"]), _ptr(out["nhits"]), _ptr(out["chi2"]), _ptr(out["state"]),
                                         _ptr(out["cov"]), _ptr(out["status"]), _ptr(ws), ws.numel(),
                                         ctypes.byref(ms), _stream(stream))
    _check(rc, "kf_autotune_find")
    return tuned, ms.value


def autotune_fit(geom: Geometry, hits, hit_surface, track_hits, stream=None):
    """Time every block size of the fit on these tracks; returns (block_threads, best ms)."""
    out = fit_tracks(geom, hits, hit_surface, track_hits, stream=stream)
    blk, ms = ctypes.c_int(), ctypes.c_float()
    lmax, n = track_hits.shape
    rc = load_library().kf_autotune_fit(geom.ref, _ptr(hits), _ptr(hit_surface), _ptr(track_hits), n, lmax,
                                        _ptr(out["state"]), _ptr(out["cov"]), _ptr(out["chi2"]), _ptr(out["ndof"]),
                                        _ptr(out["status"]), ctypes.byref(blk), ctypes.byref(ms), _stream(stream))
    _check(rc, "kf_autotune_fit")
    return blk.value, ms.value


def save_tuning(path: str, entry: dict):
    """Append an autotuning result to a JSON cache keyed by workload name and device."""
    import json
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[entry["key"]] = entry
    with open(path, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
