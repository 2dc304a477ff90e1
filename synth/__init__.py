"""Seeded synthetic events for the Kalman-filter tracking workloads.

Shared by the FP64 oracle's tests and the CUDA path's tests and benchmark. This module only
creates inputs: helix tracks from the origin in a uniform solenoid field, their exact crossings
with barrel cylinders and endcap disks, Highland multiple-scattering kicks, Gaussian hit
smearing and uniform noise hits (native code in ``synth.cpp``). It holds none of the track
fit's arithmetic.

The paper's own inputs (simulated ttbar events at pileup 50/70 in the Phase-I CMS geometry,
Sec. 3 and Sec. 4) are not available; the named workloads below stand in for them. The field
value 3.8 T is the one the paper uses (Sec. 4).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsynth.so")
_lib = None
_lock = threading.Lock()


def build_native(force: bool = False) -> str:
    """Compile ``synth.cpp`` into ``_build/libsynth.so`` (host C++, portable flags)."""
    src = os.path.join(_HERE, "synth.cpp")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, src, "-lpthread"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _SynthSurface(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("r_or_z", ctypes.c_double), ("lo", ctypes.c_double),
                ("hi", ctypes.c_double), ("x_over_x0", ctypes.c_double)]


class _SynthParams(ctypes.Structure):
    _fields_ = [("n_events", ctypes.c_int), ("tracks_lo", ctypes.c_int), ("tracks_hi", ctypes.c_int),
                ("pt_lo", ctypes.c_double), ("pt_hi", ctypes.c_double), ("eta_max", ctypes.c_double),
                ("bz", ctypes.c_double), ("sigma_rphi", ctypes.c_double), ("sigma_2nd", ctypes.c_double),
                ("noise_frac", ctypes.c_double), ("seed", ctypes.c_uint64), ("ms_on", ctypes.c_int),
                ("smear_on", ctypes.c_int), ("record_truth", ctypes.c_int), ("n_threads", ctypes.c_int),
                ("material", ctypes.c_void_p), ("eloss", ctypes.c_double), ("mass", ctypes.c_double),
                ("overlap_frac", ctypes.c_double), ("field_z2", ctypes.c_double), ("field_r2", ctypes.c_double)]


MAT_NODES = 8  # material map nodes per surface


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build_native())
            lib.synth_generate.restype = ctypes.c_void_p
            lib.synth_generate.argtypes = [ctypes.POINTER(_SynthParams), ctypes.POINTER(_SynthSurface),
                                           ctypes.c_int, ctypes.c_int]
            lib.synth_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_longlong)]
            lib.synth_copy.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 12
            lib.synth_free.argtypes = [ctypes.c_void_p]
            lib.synth_cross.restype = ctypes.c_int
            lib.synth_cross.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
            _lib = lib
    return _lib


# --------------------------------------------------------------------------------------------
# Geometry and workloads
# --------------------------------------------------------------------------------------------

BARREL, DISK = 0, 1


@dataclass(frozen=True)
class Surface:
    """One detection surface: a barrel cylinder (radius, z extent) or a disk (z, r extent)."""
    type: int
    r_or_z: float
    lo: float
    hi: float
    x_over_x0: float
    n_phi: int = 64
    n_2nd: int = 32


@dataclass(frozen=True)
class Workload:
    """A named synthetic workload: geometry, particle laws, occupancy and finder settings."""
    name: str
    surfaces: tuple
    n_events: int
    tracks_lo: int
    tracks_hi: int
    seed: int
    bz: float = 3.8
    pt_lo: float = 0.5
    pt_hi: float = 10.0
    eta_max: float = 1.0
    sigma_rphi: float = 0.01
    sigma_2nd: float = 0.1
    noise_frac: float = 0.0
    ms_on: bool = True
    chi2_cut: float = 30.0
    k_max: int = 6
    max_miss: int = 1
    # prior standard deviations at the first hit: u (transverse, cm), z or r (cm), kappa (1/GeV),
    # phi (rad), theta (rad); chosen broad compared with one hit and with scattering
    prior: tuple = (0.1, 1.0, 0.5, 0.05, 0.05)
    # material map (per surface, MAT_NODES values of x/X0 spread evenly over its extent; None: each
    # surface's x_over_x0) and mean energy loss (GeV per unit x/X0; 0: none) of a particle of mass
    # `mass` GeV (charged pion)
    material: tuple = None
    eloss: float = 0.0
    mass: float = 0.13957
    # module overlaps: probability that a crossing leaves a second hit of the particle on the
    # surface; seeds from every combination of a track's hits on its first three surfaces
    overlap_frac: float = 0.0
    combinatorial_seeds: bool = False
    # non-uniform solenoid field Bz(r, z) = bz (1 + field_z2 z^2 + field_r2 r^2), cm^-2 (0, 0: uniform)
    field_z2: float = 0.0
    field_r2: float = 0.0

    @property
    def lmax(self) -> int:
        nb = sum(1 for s in self.surfaces if s.type == BARREL)
        nd = sum(1 for s in self.surfaces if s.type == DISK)
        return nb + nd // 2 if nd else nb


def barrel_layers(n: int, r0: float = 4.0, dr: float = 4.0, half_length=None, eta_max: float = 1.0,
                  x_over_x0: float = 0.02, n_phi: int = 64, n_z: int = 32) -> list:
    """Barrel cylinders at r0, r0+dr, ...; default half-length 1.2 r sinh(eta_max) per layer, so
    every track with |eta| <= eta_max crosses every layer within the layer's z extent."""
    out = []
    for i in range(n):
        r = r0 + dr * i
        h = half_length if half_length is not None else 1.2 * r * math.sinh(eta_max)
        out.append(Surface(BARREL, r, -h, h, x_over_x0, n_phi, n_z))
    return out


def endcap_disks(n_per_side: int = 9, z0: float = 30.0, dz: float = 11.25, r_lo: float = 4.0, r_hi: float = 68.0,
                 x_over_x0: float = 0.02, n_phi: int = 64, n_r: int = 32) -> list:
    out = []
    for sign in (+1, -1):
        for j in range(n_per_side):
            out.append(Surface(DISK, sign * (z0 + dz * j), r_lo, r_hi, x_over_x0, n_phi, n_r))
    return out


def _wl_fit_small() -> Workload:
    return Workload("fit_1k_10layers", tuple(barrel_layers(10, x_over_x0=0.0)), n_events=1, tracks_lo=1000,
                    tracks_hi=1000, seed=1, ms_on=False)


def _wl_fit_batched() -> Workload:
    return Workload("fit_100ev_uneven_17layers_ms", tuple(barrel_layers(17)), n_events=100, tracks_lo=2000,
                    tracks_hi=20000, seed=2)


def _wl_find() -> Workload:
    return Workload("find_20x5k_17layers_noise30", tuple(barrel_layers(17)), n_events=20, tracks_lo=5000,
                    tracks_hi=5000, seed=3, noise_frac=0.3, k_max=6)


def _wl_learned() -> Workload:
    return Workload("learned_find_100ev_uneven_17layers", tuple(barrel_layers(17)), n_events=100,
                    tracks_lo=2000, tracks_hi=20000, seed=4, k_max=6)


def _wl_hi_occ() -> Workload:
    surf = barrel_layers(17, half_length=29.0, eta_max=2.4) + endcap_disks()
    return Workload("find_200ev_barrel_disks_noise100", tuple(surf), n_events=200, tracks_lo=3000,
                    tracks_hi=8000, seed=5, eta_max=2.4, noise_frac=1.0, k_max=8)


def steering_tables(wl, eta_barrel: float, eta_endcap: float, endcap_barrels=None) -> dict:
    """Tracking-region steering lists for a workload's geometry (regions in eta: 0 barrel, 1/2 +z/-z
    transition, 3/4 +z/-z endcap). Barrel: the barrel layers by radius; transition: the barrel
    layers by radius, then that side's disks by |z|; endcap: the innermost `endcap_barrels` barrel
    layers (all when None), then that side's disks by |z|. The region edges in eta become the FP32
    slopes c = sinh(eta) of |z| against rho. Configuration only: the finder and the oracle apply
    the lists."""
    surf = wl.surfaces
    barrels = sorted((i for i, s in enumerate(surf) if s.type == BARREL), key=lambda i: surf[i].r_or_z)
    pos = sorted((i for i, s in enumerate(surf) if s.type == DISK and s.r_or_z > 0), key=lambda i: surf[i].r_or_z)
    neg = sorted((i for i, s in enumerate(surf) if s.type == DISK and s.r_or_z < 0), key=lambda i: -surf[i].r_or_z)
    eb = barrels if endcap_barrels is None else barrels[:endcap_barrels]
    return {"c_barrel": float(np.float32(math.sinh(eta_barrel))), "c_endcap": float(np.float32(math.sinh(eta_endcap))),
            "lists": [barrels, barrels + pos, barrels + neg, eb + pos, eb + neg]}


def material_map(surfaces, x_over_x0: float = 0.02, end_factor: float = 2.0) -> tuple:
    """A synthetic r-z material map (the CMS tables are not available): on each barrel layer x/X0
    grows from x_over_x0 at z = 0 to (1 + end_factor) x_over_x0 at the layer ends (services), on
    each disk it grows likewise from the inner to the outer radius."""
    out = []
    for s in surfaces:
        nodes = []
        for k in range(MAT_NODES):
            v = s.lo + (s.hi - s.lo) * k / (MAT_NODES - 1)
            u = abs(v) / max(abs(s.lo), abs(s.hi)) if s.type == BARREL else (v - s.lo) / (s.hi - s.lo)
            nodes.append(x_over_x0 * (1.0 + end_factor * u * u))
        out.append(tuple(nodes))
    return tuple(out)


def _wl_material() -> Workload:
    surf = tuple(barrel_layers(17))
    # mean ionisation loss of a minimum-ionising particle in silicon: 3.87 MeV/cm over X0 = 9.37 cm
    return Workload("fit_100ev_17layers_material_eloss", surf, n_events=100, tracks_lo=2000, tracks_hi=20000,
                    seed=6, material=material_map(surf), eloss=0.0363)


def _wl_duplicates() -> Workload:
    return Workload("find_20x5k_17layers_overlaps30_noise30", tuple(barrel_layers(17)), n_events=20, tracks_lo=5000,
                    tracks_hi=5000, seed=7, noise_frac=0.3, k_max=6, overlap_frac=0.3, combinatorial_seeds=True)


def _wl_field() -> Workload:
    surf = barrel_layers(17, half_length=29.0, eta_max=2.4) + endcap_disks()
    # Bz falls by 5.8% from the centre to |z| = 120 cm and by 0.5% to r = 68 cm
    return Workload("find_20ev_barrel_disks_field_map", tuple(surf), n_events=20, tracks_lo=3000, tracks_hi=8000,
                    seed=8, eta_max=2.4, noise_frac=1.0, k_max=8, field_z2=-4e-6, field_r2=-1e-6)


WORKLOADS = {
    "fit_small": _wl_fit_small(),
    "fit_batched": _wl_fit_batched(),
    "find": _wl_find(),
    "learned": _wl_learned(),
    "hi_occ": _wl_hi_occ(),
    "material": _wl_material(),
    "duplicates": _wl_duplicates(),
    "field": _wl_field(),
}


def workload(name: str, **overrides) -> Workload:
    wl = WORKLOADS[name]
    return replace(wl, **overrides) if overrides else wl


# --------------------------------------------------------------------------------------------
# Event batches
# --------------------------------------------------------------------------------------------

@dataclass
class EventBatch:
    """Generated events. Hits are grouped by (event, surface): ``slab_offsets[e*n_surf+s]`` is
    the first global hit id of surface ``s`` in event ``e``. Hit ids are global indices."""
    wl: Workload
    hits: np.ndarray          # [n_hits, 2] float32: (phi, z) on barrels, (phi, r) on disks
    hit_surface: np.ndarray   # [n_hits] int32
    hit_sim: np.ndarray       # [n_hits] int32, global track id or -1 for noise
    slab_offsets: np.ndarray  # [n_events*n_surf + 1] int64
    track_event: np.ndarray   # [n_tracks] int32
    track_q: np.ndarray       # [n_tracks] int32
    track_init: np.ndarray    # [n_tracks, 3] float64: pt, eta, phi at the origin
    track_nhits: np.ndarray   # [n_tracks] int32
    track_hits: np.ndarray    # [n_tracks, lmax] int32 in path order, -1 padded
    track_surf: np.ndarray    # [n_tracks, lmax] int32
    truth_in: np.ndarray = None   # [n_tracks, lmax, 6] true (x,y,z,kappa,phi,theta) arriving
    truth_out: np.ndarray = None  # same, after the scattering kick at that surface
    extra: dict = field(default_factory=dict)

    @property
    def n_hits(self) -> int:
        return int(self.hits.shape[0])

    @property
    def n_tracks(self) -> int:
        return int(self.track_event.shape[0])

    @property
    def n_events(self) -> int:
        return int(self.wl.n_events)

    @property
    def n_surf(self) -> int:
        return len(self.wl.surfaces)

    def select_events(self, events) -> "EventBatch":
        """The sub-batch of the given events (ascending indices): their hits, tracks and truth,
        with hit ids, track ids and event numbers renumbered in the sub-batch (a rank's share of a
        fixed batch under strong scaling). Re-indexing only."""
        events = np.asarray(events, dtype=np.int64)
        if events.size > 1 and np.any(np.diff(events) <= 0):
            raise ValueError("events must be ascending and distinct")
        ns = self.n_surf
        so = self.slab_offsets.astype(np.int64)
        parts, new_so, base = [], [0], 0
        for e in events:
            a, b = so[e * ns], so[(e + 1) * ns]
            parts.append(np.arange(a, b, dtype=np.int64))
            new_so.extend((base + so[e * ns + 1:(e + 1) * ns + 1] - a).tolist())
            base += b - a
        hit_idx = np.concatenate(parts) if parts else np.zeros(0, np.int64)
        new_hit = np.full(self.n_hits + 1, -1, np.int64)  # last entry maps the -1 padding
        new_hit[hit_idx] = np.arange(hit_idx.size)
        tsel = np.nonzero(np.isin(self.track_event, events))[0]
        new_trk = np.full(self.n_tracks + 1, -1, np.int64)
        new_trk[tsel] = np.arange(tsel.size)
        th = self.track_hits[tsel]
        sim = self.hit_sim[hit_idx]
        wl = replace(self.wl, n_events=int(events.size))
        pick = (lambda a: None if a is None else a[tsel])
        return EventBatch(
            wl=wl, hits=np.ascontiguousarray(self.hits[hit_idx]), hit_surface=self.hit_surface[hit_idx].copy(),
            hit_sim=new_trk[np.where(sim >= 0, sim, self.n_tracks)].astype(np.int32),
            slab_offsets=np.asarray(new_so, dtype=np.int64),
            track_event=np.searchsorted(events, self.track_event[tsel]).astype(np.int32),
            track_q=self.track_q[tsel].copy(), track_init=self.track_init[tsel].copy(),
            track_nhits=self.track_nhits[tsel].copy(),
            track_hits=new_hit[np.where(th >= 0, th, self.n_hits)].astype(np.int32),
            track_surf=self.track_surf[tsel].copy(), truth_in=pick(self.truth_in), truth_out=pick(self.truth_out))

    def seeds(self, min_hits: int = 3, combinations: bool = None):
        """Seeds: (seed_hits [n,3], seed_track [n]). One per track from its first three true hits,
        or (combinations, the workload's default) one per combination of the track's hits on its
        first three surfaces (overlap hits included), seeds of a track consecutive, in
        lexicographic order of hit ids."""
        if combinations is None:
            combinations = getattr(self.wl, "combinatorial_seeds", False)
        ok = np.nonzero(self.track_nhits >= min_hits)[0].astype(np.int32)
        if not combinations:
            return np.ascontiguousarray(self.track_hits[ok, :3]), ok
        ns = self.n_surf
        sig = np.nonzero(self.hit_sim >= 0)[0]
        key = self.hit_sim[sig].astype(np.int64) * ns + self.hit_surface[sig]
        order = np.lexsort((sig, key))
        sk, sh = key[order], sig[order]
        lists = []
        for k in range(3):
            kk = ok.astype(np.int64) * ns + self.track_surf[ok, k]
            lo = np.searchsorted(sk, kk, side="left")
            hi = np.searchsorted(sk, kk, side="right")
            lists.append((lo, hi - lo))
        counts = lists[0][1] * lists[1][1] * lists[2][1]
        n = int(counts.sum())
        out = np.empty((n, 3), np.int32)
        trk = np.repeat(ok, counts)
        start = np.concatenate([[0], np.cumsum(counts)[:-1]])
        for t_i in range(len(ok)):  # a handful of combinations per track
            c = start[t_i]
            for a in range(lists[0][1][t_i]):
                for b in range(lists[1][1][t_i]):
                    for d in range(lists[2][1][t_i]):
                        out[c] = (sh[lists[0][0][t_i] + a], sh[lists[1][0][t_i] + b], sh[lists[2][0][t_i] + d])
                        c += 1
        return out, trk.astype(np.int32)


def generate(wl, *, n_events: int = None, seed: int = None, smear: bool = True, ms: bool = None,
             noise_frac: float = None, record_truth: bool = False, n_threads: int = 0, **overrides) -> EventBatch:
    """Generate the events of workload ``wl`` (a name or a :class:`Workload`)."""
    if isinstance(wl, str):
        wl = WORKLOADS[wl]
    upd = dict(overrides)
    if n_events is not None:
        upd["n_events"] = n_events
    if seed is not None:
        upd["seed"] = seed
    if ms is not None:
        upd["ms_on"] = ms
    if noise_frac is not None:
        upd["noise_frac"] = noise_frac
    if upd:
        wl = replace(wl, **upd)
    lib = _load()
    # The geometry's canonical values are FP32 (the oracle and the CUDA path read FP32 geometry),
    # so the simulation uses the same rounded numbers.
    f32 = lambda v: float(np.float32(v))  # noqa: E731
    surf = (_SynthSurface * len(wl.surfaces))()
    for i, s in enumerate(wl.surfaces):
        surf[i] = _SynthSurface(s.type, f32(s.r_or_z), f32(s.lo), f32(s.hi), f32(s.x_over_x0) if wl.ms_on else 0.0)
    mat = None
    if wl.material is not None:
        mat = np.array([[f32(v) for v in nodes] for nodes in wl.material], np.float64)
        if mat.shape != (len(wl.surfaces), MAT_NODES):
            raise ValueError(f"material map must be [{len(wl.surfaces)}][{MAT_NODES}]")
    prm = _SynthParams(wl.n_events, wl.tracks_lo, wl.tracks_hi, wl.pt_lo, wl.pt_hi, wl.eta_max, f32(wl.bz),
                       wl.sigma_rphi, wl.sigma_2nd, wl.noise_frac, wl.seed, int(wl.ms_on), int(smear),
                       int(record_truth), n_threads, None if mat is None else mat.ctypes.data, f32(wl.eloss),
                       f32(wl.mass), wl.overlap_frac, f32(wl.field_z2), f32(wl.field_r2))
    lmax = wl.lmax
    h = lib.synth_generate(ctypes.byref(prm), surf, len(wl.surfaces), lmax)
    if not h:
        raise ValueError("synth_generate rejected its arguments")
    try:
        nh, nt = ctypes.c_longlong(), ctypes.c_longlong()
        lib.synth_sizes(h, ctypes.byref(nh), ctypes.byref(nt))
        nh, nt = nh.value, nt.value
        hits = np.empty((nh, 2), np.float32)
        hit_surface = np.empty(nh, np.int32)
        hit_sim = np.empty(nh, np.int32)
        slab = np.empty(wl.n_events * len(wl.surfaces) + 1, np.int64)
        track_event = np.empty(nt, np.int32)
        track_q = np.empty(nt, np.int32)
        track_init = np.empty((nt, 3), np.float64)
        track_nhits = np.empty(nt, np.int32)
        track_hits = np.empty((nt, lmax), np.int32)
        track_surf = np.empty((nt, lmax), np.int32)
        tin = np.zeros((nt, lmax, 6), np.float64) if record_truth else None
        tout = np.zeros((nt, lmax, 6), np.float64) if record_truth else None
        p = lambda a: a.ctypes.data if a is not None else None  # noqa: E731
        lib.synth_copy(h, p(hits), p(hit_surface), p(hit_sim), p(slab), p(track_event), p(track_q), p(track_init),
                       p(track_nhits), p(track_hits), p(track_surf), p(tin), p(tout))
    finally:
        lib.synth_free(h)
    return EventBatch(wl, hits, hit_surface, hit_sim, slab, track_event, track_q, track_init, track_nhits,
                      track_hits, track_surf, tin, tout)


def cross(surface_type: int, r_or_z: float, bz: float, q: int, pos, mom):
    """Exact crossing of one particle with a cylinder (type 0) or plane z = r_or_z (type 1).

    Returns (pos_out, mom_out, psi) or None when the surface is not reached; psi is the turning
    angle of the momentum in the transverse plane."""
    lib = _load()
    pos = np.ascontiguousarray(pos, np.float64)
    mom = np.ascontiguousarray(mom, np.float64)
    po = np.empty(3)
    mo = np.empty(3)
    psi = ctypes.c_double()
    rc = lib.synth_cross(surface_type, r_or_z, bz, q, pos.ctypes.data, mom.ctypes.data, po.ctypes.data,
                         mo.ctypes.data, ctypes.addressof(psi))
    if rc != 0:
        return None
    return po, mo, psi.value


def mlp_init(seed: int, n_in: int = 14, n_hid: int = 64) -> np.ndarray:
    """He-initialised weights of the learned hit-proposal MLP (n_in -> n_hid -> n_hid -> 1) as
    one float32 vector: W1[n_hid][n_in], b1, W2[n_hid][n_hid], b2, W3[n_hid], b3. Weights are
    N(0, 2 / fan_in), biases 0, drawn from numpy's PCG64 stream of ``seed``. These random numbers
    are an input of training, drawn here so that every consumer gets the same ones."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / n_in), n_hid * n_in), np.zeros(n_hid),
             rng.normal(0.0, np.sqrt(2.0 / n_hid), n_hid * n_hid), np.zeros(n_hid),
             rng.normal(0.0, np.sqrt(2.0 / n_hid), n_hid), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)
