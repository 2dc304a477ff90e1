"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Bars: hit index and bin lookup bit-exact; fitted parameters within 1e-4 relative and chi2 within
1e-3 relative; finding hit assignments identical on >= 99.9% of seeds with efficiency equal within
0.1%. Relative tolerances use a floor scale per quantity (1 cm for positions, 0.1/GeV for kappa,
1 rad for angles, 1 for chi2) so values near zero are compared on the scale of the quantity.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

FLOOR = np.array([1.0, 1.0, 1.0, 0.1, 1.0, 1.0])


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as k
    k.load_library()
    return k


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _state_rel_err(p_gpu, p_ora):
    d = p_gpu.astype(np.float64) - p_ora
    d[:, 4] = _wrap(d[:, 4])
    return np.abs(d) / np.maximum(np.abs(p_ora), FLOOR)


def _index_both(kf, wl, b):
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    torch.cuda.synchronize()
    off, sh, si, sub = oracle.build_index(oracle.Geometry(wl), b.hits, b.slab_offsets, b.n_events, with_sub=True)
    return idx, (off, sh, si, sub), dev, g


@pytest.mark.parametrize("wl_name,n_ev,nt", [("find", 3, 2500), ("hi_occ", 2, 1500), ("fit_batched", 2, 20000)])
def test_hit_index_bit_exact(kf, wl_name, n_ev, nt):
    wl = synth.workload(wl_name, n_events=n_ev, tracks_lo=nt // 2, tracks_hi=nt)
    b = synth.generate(wl)
    idx, (off, sh, si, sub), _, _ = _index_both(kf, wl, b)
    assert np.array_equal(idx.bin_off.cpu().numpy(), off.astype(np.int32))
    assert np.array_equal(idx.sub_off.cpu().numpy().view(np.uint16), sub)
    assert np.array_equal(idx.sorted_ids.cpu().numpy(), si)
    assert np.array_equal(idx.sorted_hits.cpu().numpy().view(np.uint32), sh.view(np.uint32))
    # search records: (cos phi, sin phi) to FP32 accuracy, the second coordinate and the id exact
    rec = idx.sorted_rec.cpu().numpy()
    d = rec[:, :2].astype(np.float64)
    ph = sh[:, 0].astype(np.float64)
    assert np.abs(d[:, 0] - np.cos(ph)).max() < 3e-7 and np.abs(d[:, 1] - np.sin(ph)).max() < 3e-7
    assert np.array_equal(rec[:, 2].view(np.uint32), sh[:, 1].view(np.uint32))
    assert np.array_equal(rec[:, 3].view(np.int32), si)


def test_hit_index_edge_cases(kf):
    """Empty slabs, a single hit, hits on bin edges, at +-pi and outside the z extent."""
    wl = synth.workload("find", n_events=2, tracks_lo=3, tracks_hi=3)
    b = synth.generate(wl)
    # keep only surface 0 hits of event 0 plus edge values, everything else empty
    s0 = wl.surfaces[0]
    edge = np.array([[-np.pi, s0.lo], [np.float32(np.pi), s0.hi], [0.0, 0.0], [np.nextafter(np.float32(np.pi), 0), -1e3],
                     [-np.float32(np.pi), 1e3], [0.5, s0.lo + (s0.hi - s0.lo) / 32]], np.float32)
    hits = np.concatenate([b.hits[b.slab_offsets[0]:b.slab_offsets[1]], edge]).astype(np.float32)
    n = hits.shape[0]
    slab = np.full(b.n_events * b.n_surf + 1, n, np.int64)
    slab[0] = 0
    b.hits, b.slab_offsets = hits, slab
    b.hit_surface = np.zeros(n, np.int32)
    idx, (off, sh, si, sub), _, _ = _index_both(kf, wl, b)
    assert np.array_equal(idx.bin_off.cpu().numpy(), off.astype(np.int32))
    assert np.array_equal(idx.sub_off.cpu().numpy().view(np.uint16), sub)
    assert np.array_equal(idx.sorted_ids.cpu().numpy(), si)


def test_hit_index_crowded_slab_at_capacity(kf):
    """One slab of exactly the compiled capacity (KF_MAX_SLAB_HITS hits): a quarter of them in one
    bin, 1,000 at identical coordinates (same bin and sub-bin, ordered by id alone), the rest
    uniform; every other slab empty."""
    wl = synth.workload("find", n_events=1, tracks_lo=3, tracks_hi=3)
    b = synth.generate(wl)
    s0 = wl.surfaces[0]
    n = kf.KF_MAX_SLAB_HITS
    rng = np.random.default_rng(11)
    phi = rng.uniform(-np.pi, np.pi, n)
    z = rng.uniform(s0.lo, s0.hi, n)
    k = n // 4
    phi[:k] = 0.01 + rng.uniform(0.0, 1e-3, k)
    z[:k] = s0.lo + 1e-3
    phi[k:k + 1000] = 0.02
    z[k:k + 1000] = s0.lo + 0.5
    perm = rng.permutation(n)
    hits = np.stack([phi[perm], z[perm]], axis=1).astype(np.float32)
    slab = np.full(b.n_events * b.n_surf + 1, n, np.int64)
    slab[0] = 0
    b.hits, b.slab_offsets = hits, slab
    b.hit_surface = np.zeros(n, np.int32)
    idx, (off, sh, si, sub), dev, _ = _index_both(kf, wl, b)
    assert dev["max_slab_hits"] == n
    assert np.array_equal(idx.bin_off.cpu().numpy(), off.astype(np.int32))
    assert np.array_equal(idx.sub_off.cpu().numpy().view(np.uint16), sub)
    assert np.array_equal(idx.sorted_ids.cpu().numpy(), si)
    assert np.array_equal(idx.sorted_hits.cpu().numpy().view(np.uint32), sh.view(np.uint32))


def test_hit_index_empty_event(kf):
    wl = synth.workload("find", n_events=1, tracks_lo=0, tracks_hi=0)
    b = synth.generate(wl)
    assert b.n_hits == 0
    g = kf.Geometry(wl)
    hits = torch.zeros((0, 2), dtype=torch.float32, device="cuda")
    slab = torch.zeros(b.n_surf + 1, dtype=torch.int32, device="cuda")
    idx = kf.HitIndex(g, 1, 1)
    kf.build_hit_index(g, hits, slab, 1, 0, index=idx)
    assert int(idx.bin_off.abs().sum()) == 0


def _fit_both(kf, wl, b, tracks=None):
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    th = b.track_hits if tracks is None else tracks
    out = kf.fit_tracks(g, dev["hits"], dev["hit_surface"], torch.from_numpy(np.ascontiguousarray(th.T)).cuda())
    torch.cuda.synchronize()
    r = oracle.fit(oracle.Geometry(wl), b.hits, b.hit_surface, th)
    # surface type at each track's last hit (the covariance's null direction depends on it)
    last = np.array([row[row >= 0][-1] if (row >= 0).any() else 0 for row in th])
    r["surf_type"] = np.array([wl.surfaces[s].type == synth.DISK for s in b.hit_surface[last]])
    return {k: v.cpu().numpy() for k, v in out.items()}, r


def _assert_fit_parity(gpu, ora):
    assert np.array_equal(gpu["status"], ora["status"])
    assert np.array_equal(gpu["ndof"], ora["ndof"])
    ok = ora["status"] == 0
    rel = _state_rel_err(gpu["state"].T[ok], ora["p"][ok])
    assert rel.max() < 1e-4, rel.max(axis=0)
    c2r = np.abs(gpu["chi2"][ok] - ora["chi2"][ok]) / np.maximum(ora["chi2"][ok], 1.0)
    assert c2r.max() < 1e-3, c2r.max()
    _assert_cov_parity(gpu["cov"].T[ok], ora["cov"][ok], ora["p"][ok], ora["surf_type"][ok])


def _tangent_basis(p, disk):
    """Orthonormal basis of the 5D tangent space: complement of the surface normal (the
    covariance is singular along the normal by construction)."""
    n = np.zeros(6)
    if disk:
        n[2] = 1.0
    else:
        n[:2] = p[:2] / np.hypot(p[0], p[1])
    q, _ = np.linalg.qr(np.column_stack([n, np.eye(6)]))
    return q[:, 1:6]


def _assert_cov_parity(cov_gpu, cov_ora, p_ora, disk=None, tol=1e-3):
    """Tangent-space covariance elements agree within tol of sqrt(A_ii A_jj)."""
    C = oracle.unpack_cov(cov_ora)
    Cg = oracle.unpack_cov(cov_gpu.astype(np.float64))
    worst = 0.0
    for t in range(C.shape[0]):
        T = _tangent_basis(p_ora[t], bool(disk[t]) if disk is not None else False)
        A, Ag = T.T @ C[t] @ T, T.T @ Cg[t] @ T
        d = np.sqrt(np.diag(A))
        worst = max(worst, (np.abs(Ag - A) / np.outer(d, d)).max())
    assert worst < tol, worst


def test_fit_parity_small(kf):
    """1000 tracks, 10 layers, no scattering (the small fitting workload)."""
    wl = synth.workload("fit_small")
    b = synth.generate(wl)
    gpu, ora = _fit_both(kf, wl, b)
    _assert_fit_parity(gpu, ora)


@pytest.mark.parametrize("wl_name", ["fit_batched", "hi_occ", "material"])
def test_seed_states_parity(kf, wl_name):
    """kf_seed_states (the seed fit alone) against the oracle's fit of the three seed hits: the
    state, covariance and chi2 at hit 3; seeds with an invalid hit or event are marked failed."""
    wl = synth.workload(wl_name, n_events=2, tracks_lo=1500, tracks_hi=3000)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    sh, st = b.seeds()
    sh = sh.copy()
    ev = b.track_event[st].astype(np.int32)
    bad = np.arange(0, len(st), 97)
    sh[bad[::2], 1] = -1           # a missing hit
    ev[bad[1::2]] = b.n_events     # an event outside the batch
    state, surf = kf.seed_states(g, dev["hits"], dev["hit_surface"], torch.from_numpy(np.ascontiguousarray(sh.T)).cuda(),
                                 torch.from_numpy(ev).cuda(), b.n_events)
    torch.cuda.synchronize()
    state, surf = state.cpu().numpy(), surf.cpu().numpy()
    failed = state[27] < 0
    assert failed[bad].all()
    good = np.ones(len(st), bool)
    good[bad] = False
    r = oracle.fit(oracle.Geometry(wl), b.hits, b.hit_surface, sh[good])
    assert np.array_equal(failed[good], r["status"] != 0)  # the same seeds fail on both sides
    ok = good & ~failed
    r = {k: v[r["status"] == 0] for k, v in r.items()}
    # The fit bars (1e-4 relative on the state, 1e-3 on chi2) hold for 99% of the seeds; a seed
    # whose three hits are close in the transverse plane (consecutive disks at high |eta|) has an
    # ill-conditioned curvature, where FP32 rounding shows up to ~1e-3 relative in kappa. Every
    # seed's positions meet the bar, and its kappa, phi and theta stay within 1e-2 of their own
    # standard deviations (windows are sqrt(30) standard deviations wide, so that moves no hit
    # decision in practice).
    rel = _state_rel_err(state[:6, ok].T, r["p"])
    assert (rel.max(axis=1) < 1e-4).mean() >= 0.99, rel.max(axis=0)
    assert rel[:, :3].max() < 1e-4, rel[:, :3].max(axis=0)  # positions: every seed
    sig = np.sqrt(np.diagonal(oracle.unpack_cov(r["cov"]), axis1=1, axis2=2))[:, 3:]
    dp = state[3:6, ok].T.astype(np.float64) - r["p"][:, 3:]
    dp[:, 1] = _wrap(dp[:, 1])
    pulls = np.abs(dp) / sig  # kappa, phi, theta in units of their standard deviations
    assert pulls.max() < 1e-2, pulls.max(axis=0)
    c2r = np.abs(state[27, ok] - r["chi2"]) / np.maximum(r["chi2"], 1.0)
    assert (c2r < 1e-3).mean() >= 0.99 and c2r.max() < 1e-2, c2r.max()
    disk = np.array([wl.surfaces[s_].type == synth.DISK for s_ in b.hit_surface[sh[ok, 2]]])
    _assert_cov_parity(state[6:27, ok].T, r["cov"], r["p"], disk)
    assert np.array_equal(surf[ok], b.hit_surface[sh[ok, 2]])


def test_fit_parity_scattering_and_disks(kf):
    for name in ("fit_batched", "hi_occ"):
        wl = synth.workload(name, n_events=2, tracks_lo=1500, tracks_hi=3000)
        b = synth.generate(wl)
        gpu, ora = _fit_both(kf, wl, b)
        _assert_fit_parity(gpu, ora)


def test_fit_parity_material_map_and_energy_loss(kf):
    """Material map + mean energy loss, with and without scattering."""
    for ms in (True, False):
        wl = synth.workload("material", n_events=2, tracks_lo=1500, tracks_hi=3000, ms_on=ms)
        b = synth.generate(wl)
        gpu, ora = _fit_both(kf, wl, b)
        _assert_fit_parity(gpu, ora)


def test_find_parity_material_map_and_energy_loss(kf):
    wl = synth.workload("material", n_events=2, tracks_lo=1500, tracks_hi=2500, noise_frac=0.3)
    b = synth.generate(wl)
    gpu, ora, st = _find_both(kf, wl, b)
    _assert_find_parity(b, gpu, ora, st)


def test_fit_parity_field_map(kf):
    """Parametrised solenoid field on the barrel + disk geometry (|eta| < 2.4), with and without
    scattering."""
    for ms in (True, False):
        wl = synth.workload("field", n_events=2, tracks_lo=1500, tracks_hi=3000, ms_on=ms)
        b = synth.generate(wl)
        gpu, ora = _fit_both(kf, wl, b)
        _assert_fit_parity(gpu, ora)


def test_find_parity_field_map(kf):
    wl = synth.workload("field", n_events=2, tracks_lo=800, tracks_hi=1500)
    b = synth.generate(wl)
    gpu, ora, st = _find_both(kf, wl, b)
    _assert_find_parity(b, gpu, ora, st)


def test_find_and_fit_parity_with_every_option_at_once(kf):
    """Field map, material map, energy loss and region steering together on the barrel + disk
    geometry (the general finder kernel with all its branches live)."""
    import dataclasses
    base = synth.workload("field", n_events=2, tracks_lo=800, tracks_hi=1500)
    wl = dataclasses.replace(base, material=synth.material_map(base.surfaces), eloss=0.0363)
    b = synth.generate(wl)
    gpu, ora, st = _find_both(kf, wl, b, steering=_steering_without(wl, ()))
    _assert_find_parity(b, gpu, ora, st)
    gpu_f, ora_f = _fit_both(kf, wl, b)
    _assert_fit_parity(gpu_f, ora_f)


def test_field_coefficients_rejected_when_not_finite(kf):
    import dataclasses
    wl = synth.workload("field", n_events=1, tracks_lo=50, tracks_hi=50)
    b = synth.generate(wl)
    dev = kf.to_device_event_batch(b)
    with pytest.raises(kf.KfError):
        g = kf.Geometry(dataclasses.replace(wl, field_z2=float("nan")))
        kf.fit_tracks(g, dev["hits"], dev["hit_surface"], dev["track_hits"])


def test_fit_with_misses_and_short_tracks(kf):
    """-1 entries inside a list are skipped; lists with fewer than three seed hits are rejected."""
    wl = synth.workload("fit_batched", n_events=1, tracks_lo=700, tracks_hi=700)
    b = synth.generate(wl)
    th = b.track_hits.copy()
    rng = np.random.default_rng(0)
    for t in range(th.shape[0]):
        k = rng.integers(3, th.shape[1], size=2)
        th[t, k] = -1
    th[:5, 1] = -1
    gpu, ora = _fit_both(kf, wl, b, th)
    assert np.all(ora["status"][:5] == 3)
    _assert_fit_parity(gpu, ora)


def _find_both(kf, wl, b, **kw):
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    prm = kf.find_params(kw.get("chi2_cut", wl.chi2_cut), kw.get("k_max", wl.k_max), kw.get("max_miss", wl.max_miss),
                         wl.lmax, steering_tables=kw.get("steering"))
    out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    torch.cuda.synchronize()
    sh, st = b.seeds()
    r = oracle.find(oracle.Geometry(wl), b, sh, b.track_event[st], **kw)
    gpu = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    return gpu, r, st


def _assert_find_parity(b, gpu, ora, st):
    same = (gpu["hits"].T == ora["hits"]).all(axis=1)
    assert same.mean() >= 0.999, same.mean()
    assert np.array_equal(gpu["status"], ora["status"])
    e_g = oracle.efficiency(b, st, gpu["hits"].T, gpu["nhits"])[0]
    e_o = oracle.efficiency(b, st, ora["hits"], ora["n_hits"])[0]
    assert abs(e_g - e_o) <= 0.001
    # identical tracks carry the same fit
    ok = same & (ora["status"] == 0)
    _assert_track_state_parity(gpu["state"].T[ok], gpu["chi2"][ok], ora["p"][ok], ora["cov"][ok], ora["chi2"][ok])


def _assert_track_state_parity(p_gpu, chi2_gpu, p_ora, cov_ora, chi2_ora):
    """Tracks with identical hit lists carry the fit bars on every track: 1e-4 relative on the
    state, 1e-3 on chi2 (measured maxima over the test workloads: 4e-5 and 2.3e-4); kappa, phi and
    theta also within 1e-2 of their own standard deviations (measured: 2e-3)."""
    rel = _state_rel_err(p_gpu, p_ora)
    worst = rel.max(axis=1)
    print(f"state: max {worst.max():.2e}, 99.9% {np.quantile(worst, 0.999):.2e}")
    assert worst.max() < 1e-4, rel.max(axis=0)
    sig = np.sqrt(np.diagonal(oracle.unpack_cov(cov_ora), axis1=1, axis2=2))[:, 3:]
    dp = p_gpu[:, 3:].astype(np.float64) - p_ora[:, 3:]
    dp[:, 1] = _wrap(dp[:, 1])
    pulls = np.abs(dp) / sig
    print(f"kappa, phi, theta in sigma: max {pulls.max(axis=0)}")
    assert pulls.max() < 1e-2, pulls.max(axis=0)
    c2r = np.abs(chi2_gpu - chi2_ora) / np.maximum(chi2_ora, 1.0)
    print(f"chi2: max {c2r.max():.2e}, 99.9% {np.quantile(c2r, 0.999):.2e}")
    assert c2r.max() < 1e-3, c2r.max()


@pytest.mark.parametrize("wl_name,n_ev,nt,k", [("find", 2, 2500, 6), ("find", 2, 2500, 1), ("hi_occ", 2, 1500, 8),
                                              ("learned", 2, 3000, 16)])
def test_find_parity(kf, wl_name, n_ev, nt, k):
    wl = synth.workload(wl_name, n_events=n_ev, tracks_lo=nt // 2, tracks_hi=nt)
    b = synth.generate(wl)
    gpu, ora, st = _find_both(kf, wl, b, k_max=k)
    _assert_find_parity(b, gpu, ora, st)


def _steering_without(wl, surfaces):
    tab = synth.steering_tables(wl, 0.4, 1.8, endcap_barrels=3)
    tab["lists"] = [[x for x in lst if x not in surfaces] for lst in tab["lists"]]
    return tab


@pytest.mark.parametrize("dropped", [(), (6, 20)])
def test_find_parity_region_steering(kf, dropped):
    """Region steering on the barrel + disk geometry against the oracle: lists in crossing order,
    and lists without barrel layer 6 and the third +z disk."""
    wl = synth.workload("hi_occ", n_events=2, tracks_lo=800, tracks_hi=1500)
    b = synth.generate(wl)
    gpu, ora, st = _find_both(kf, wl, b, steering=_steering_without(wl, dropped))
    _assert_find_parity(b, gpu, ora, st)
    if dropped:
        assert not np.isin(gpu["hits"], np.nonzero(np.isin(b.hit_surface, dropped))[0]).any()


def test_region_steering_in_crossing_order_equals_geometric_rule_on_gpu(kf):
    wl = synth.workload("hi_occ", n_events=2, tracks_lo=800, tracks_hi=1500)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    outs = []
    for tab in (None, _steering_without(wl, ())):
        prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, steering_tables=tab)
        out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
        outs.append({k: v.cpu().numpy() for k, v in out.items() if k != "workspace"})
    for k in ("hits", "nhits", "status"):
        assert np.array_equal(outs[0][k], outs[1][k])


def test_region_steering_rejects_invalid_lists(kf):
    wl = synth.workload("hi_occ", n_events=1, tracks_lo=50, tracks_hi=50)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    for bad in ("duplicate", "range", "edges"):
        tab = synth.steering_tables(wl, 0.4, 1.8)
        if bad == "duplicate":
            tab["lists"][0] = tab["lists"][0] + [tab["lists"][0][0]]
        elif bad == "range":
            tab["lists"][1] = tab["lists"][1] + [len(wl.surfaces)]
        else:
            tab["c_barrel"], tab["c_endcap"] = 2.0, 1.0
        prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, steering_tables=tab)
        with pytest.raises(kf.KfError):
            kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)


def test_find_with_invalid_seeds(kf):
    """Seeds with a missing hit or an event outside the batch fail with empty outputs on both
    sides; the other seeds are unaffected."""
    wl = synth.workload("find", n_events=2, tracks_lo=600, tracks_hi=600)
    b = synth.generate(wl)
    sh, st = b.seeds()
    sh = sh.copy()
    ev = b.track_event[st].astype(np.int32).copy()
    sh[0, 0] = -1
    sh[1, 2] = -1
    ev[2] = b.n_events
    ev[3] = -1
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
    out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], torch.from_numpy(np.ascontiguousarray(sh.T)).cuda(),
                         torch.from_numpy(ev).cuda(), prm)
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}
    r = oracle.find(oracle.Geometry(wl), b, sh, ev)
    assert gpu["status"][:4].tolist() == [1, 1, 1, 1] and r["status"][:4].tolist() == [1, 1, 1, 1]
    assert np.all(gpu["hits"][:, :4] == -1) and np.all(gpu["nhits"][:4] == 0) and np.all(np.isnan(gpu["chi2"][:4]))
    _assert_find_parity(b, gpu, r, st)


def test_find_and_fit_at_the_maximum_sizes(kf):
    """31 barrel layers (lmax = KF_MAX_LMAX, the longest trace and hit list) with K = KF_MAX_K;
    one more layer is rejected."""
    import dataclasses
    wl = dataclasses.replace(synth.workload("find", n_events=1, tracks_lo=400, tracks_hi=400),
                             surfaces=tuple(synth.barrel_layers(31, dr=2.2)), k_max=kf.KF_MAX_K, noise_frac=0.3)
    assert wl.lmax == kf.KF_MAX_LMAX
    b = synth.generate(wl)
    gpu, ora, st = _find_both(kf, wl, b, k_max=kf.KF_MAX_K)
    _assert_find_parity(b, gpu, ora, st)
    assert gpu["nhits"].max() == kf.KF_MAX_LMAX
    gpu_f, ora_f = _fit_both(kf, wl, b)
    _assert_fit_parity(gpu_f, ora_f)
    big = dataclasses.replace(wl, surfaces=tuple(synth.barrel_layers(32, dr=2.1)))
    prm = kf.find_params(big.chi2_cut, big.k_max, big.max_miss, big.lmax)
    assert kf.find_workspace_size(10, prm) == 0
    bb = synth.generate(big)
    g2 = kf.Geometry(big)
    d2 = kf.to_device_event_batch(bb)
    idx2 = kf.build_hit_index(g2, d2["hits"], d2["slab_offsets"], bb.n_events, d2["max_slab_hits"])
    with pytest.raises(kf.KfError):
        kf.find_tracks(g2, idx2, d2["hits"], d2["hit_surface"], d2["seed_hits"], d2["seed_event"], prm)


def test_find_parity_dense_noise(kf):
    """Many branches per seed: 5 noise hits per signal hit."""
    wl = synth.workload("find", n_events=1, tracks_lo=1200, tracks_hi=1200, noise_frac=5.0)
    b = synth.generate(wl)
    gpu, ora, st = _find_both(kf, wl, b)
    _assert_find_parity(b, gpu, ora, st)


def test_general_and_plain_finder_instances_agree(kf):
    """A flat material map (every node at the surface's x/X0) and no energy loss select the general
    finder kernel (the one that serves steering, material map and field map) with the physics of
    the plain one: the two instances find the same tracks."""
    import dataclasses
    base = synth.workload("hi_occ", n_events=2, tracks_lo=800, tracks_hi=1500)
    flat = dataclasses.replace(base, material=tuple(tuple([s.x_over_x0] * synth.MAT_NODES) for s in base.surfaces))
    b = synth.generate(base)
    outs = []
    for wl in (base, flat):
        g = kf.Geometry(wl)
        dev = kf.to_device_event_batch(b)
        idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
        prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
        out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
        outs.append({k: v.cpu().numpy() for k, v in out.items() if k != "workspace"})
    same = (outs[0]["hits"] == outs[1]["hits"]).all(axis=0)
    assert same.mean() >= 0.9999, same.mean()  # the two compilations may round a contraction apart
    assert np.array_equal(outs[0]["status"], outs[1]["status"])
    ok = same & (outs[0]["status"] == 0)
    for k in ("chi2", "state"):
        a, c = outs[0][k][..., ok].astype(np.float64), outs[1][k][..., ok].astype(np.float64)
        assert np.all(np.abs(a - c) <= 1e-5 * np.maximum(np.abs(a), 1.0)), k


def test_autotuner_configurations_give_identical_results(kf):
    """Block size and candidate capacity change the schedule, never the result: every configuration
    the autotuner tries finds the same tracks, and it returns one of them."""
    wl = synth.workload("find", n_events=2, tracks_lo=1500, tracks_hi=2500, noise_frac=1.0)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    ref = None
    for blk in (64, 160, 256):
        for cap in (6, 8, 16):
            prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, block_threads=blk, k_capacity=cap)
            out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
            hits = out["hits"].cpu().numpy()
            if ref is None:
                ref = hits
            assert np.array_equal(hits, ref), (blk, cap)
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
    tuned, ms = kf.autotune_find(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    assert tuned.block_threads in range(64, 257, 32) and tuned.k_capacity in (6, 8) and ms > 0
    blk, ms = kf.autotune_fit(g, dev["hits"], dev["hit_surface"], dev["track_hits"])
    assert blk in range(64, 257, 32) and ms > 0


def _find_gpu(kf, wl, b, **kw):
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    prm = kf.find_params(wl.chi2_cut, kw.get("k_max", wl.k_max), wl.max_miss, wl.lmax,
                         steering_tables=kw.get("steering"), adaptive_capacity=kw.get("adaptive", 0),
                         block_threads=kw.get("block", 0))
    out = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    torch.cuda.synchronize()
    # work counters at the head of the workspace: [2] = seeds the first pass left to the second
    overflow = int(out["workspace"][8:12].view(torch.int32).item())
    return {k: v.cpu().numpy() for k, v in out.items() if k != "workspace"}, overflow


@pytest.mark.parametrize("wl_name,n_ev,k,adaptive,opts", [
    ("hi_occ", 3, 8, 4, {}), ("hi_occ", 3, 8, 2, {}), ("hi_occ", 3, 8, 4, {"block": 96}),
    ("find", 3, 6, 4, {}), ("find", 3, 16, 4, {}), ("material", 3, 6, 4, {}), ("hi_occ", 3, 8, 4, {"steer": True})])
def test_adaptive_capacity_gives_the_single_pass_results(kf, wl_name, n_ev, k, adaptive, opts):
    """Two passes (a small capacity first, its overflowing seeds again at the full capacity) give
    exactly the outputs of one pass at the full capacity, and both passes do work."""
    wl = synth.workload(wl_name, n_events=n_ev)
    b = synth.generate(wl)
    kw = {"k_max": k, "block": opts.get("block", 0)}
    if opts.get("steer"):
        kw["steering"] = synth.steering_tables(wl, 0.4, 1.8, endcap_barrels=3)
    one, ovf1 = _find_gpu(kf, wl, b, **kw)
    two, ovf2 = _find_gpu(kf, wl, b, adaptive=adaptive, **kw)
    assert ovf1 == 0
    n = one["status"].shape[0]
    assert 0 < ovf2 < n, (ovf2, n)
    for key in ("hits", "nhits", "status"):
        assert np.array_equal(one[key], two[key]), key
    for key in ("chi2", "state", "cov"):
        assert np.array_equal(one[key].view(np.uint32), two[key].view(np.uint32)), key


def test_adaptive_capacity_parity_with_the_oracle(kf):
    wl = synth.workload("hi_occ", n_events=3)
    b = synth.generate(wl)
    gpu, ovf = _find_gpu(kf, wl, b, adaptive=4)
    assert ovf > 0
    sh, st = b.seeds()
    ora = oracle.find(oracle.Geometry(wl), b, sh, b.track_event[st])
    _assert_find_parity(b, gpu, ora, st)
