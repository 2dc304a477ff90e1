"""Pins of the oracle's parametrised solenoid field (Sec. 3.1: constant or parametrised magnetic
field), CPU only.

Reading: Bz(r, z) = bz (1 + field_z2 z^2 + field_r2 r^2); a step between surfaces is a helix in
the field at the midpoint of its chord, the chord taken from the path in the field at the step's
start. The generator moves particles through the same field independently (half-centimetre helix
substeps, each in the field at its own midpoint), so its crossings test the oracle's one-step
model; a closed-form helix written here tests where the field is evaluated.
"""
import dataclasses

import numpy as np

import oracle
import synth

K_CURV = 0.00299792458


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _field(wl, x, y, z):
    bz, a, b = (float(np.float32(v)) for v in (wl.bz, wl.field_z2, wl.field_r2))
    return bz * (1.0 + a * z * z + b * (x * x + y * y))


def _helix(p, w, s):
    """Closed-form helix: transverse path s, signed curvature w."""
    x0, y0, z0, _, phi, th = p
    return np.array([x0 + (np.sin(phi + w * s) - np.sin(phi)) / w, y0 - (np.cos(phi + w * s) - np.cos(phi)) / w,
                     z0 + s / np.tan(th)])


def _path_to_radius(p, w, R):
    """Smallest s > 0 with |(x, y)(s)| = R, by bisection on a fine bracket."""
    f = lambda s: np.hypot(*_helix(p, w, s)[:2]) - R
    grid = np.linspace(1e-9, 3 * R, 3001)
    v = np.array([f(s) for s in grid])
    i = np.nonzero((v[:-1] < 0) & (v[1:] >= 0))[0][0]
    lo, hi = grid[i], grid[i + 1]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_step_uses_the_field_at_the_chord_midpoint():
    """Barrel-to-barrel steps far from z = 0 (strong field gradient) against a closed-form helix in
    the field at the midpoint of the chord; the field at the start is measurably different."""
    wl = synth.workload("field", n_events=1, tracks_lo=300, tracks_hi=300, ms_on=False, noise_frac=0.0)
    b = synth.generate(wl, smear=False, record_truth=True)
    g = oracle.Geometry(wl)
    barrel = [i for i, s in enumerate(wl.surfaces) if s.type == synth.BARREL]
    checked, far = 0, 0
    for t in range(b.n_tracks):
        for k in range(b.track_nhits[t] - 1):
            s0, s1 = int(b.track_surf[t, k]), int(b.track_surf[t, k + 1])
            p0 = b.truth_out[t, k]
            if s0 not in barrel or s1 not in barrel or abs(p0[2]) < 15.0:
                continue
            R = wl.surfaces[s1].r_or_z
            w0 = -K_CURV * _field(wl, *p0[:3]) * p0[3]
            sa = _path_to_radius(p0, w0, float(np.float32(R)))
            m = p0[:3] + 0.5 * sa * np.array([np.cos(p0[4]), np.sin(p0[4]), 1.0 / np.tan(p0[5])])
            w1 = -K_CURV * _field(wl, *m) * p0[3]
            want = _helix(p0, w1, _path_to_radius(p0, w1, float(np.float32(R))))
            got = oracle.propagate(g, p0, None, s1)
            assert got is not None
            assert np.abs(got[0][:3] - want).max() < 1e-8, (t, k, got[0][:3] - want)
            at_start = _helix(p0, w0, sa)
            far += np.abs(at_start - want).max() > 1e-6
            checked += 1
            if checked >= 25:
                break
        if checked >= 25:
            break
    assert checked >= 25 and far >= 10


def test_one_step_model_reproduces_the_generator_crossings():
    """From each true state on a surface to the next crossing: the one-step midpoint model lands
    within a few micrometres of the generator's finely stepped crossing; a uniform field misses by
    tens of micrometres."""
    wl = synth.workload("field", n_events=1, tracks_lo=500, tracks_hi=500, ms_on=False, noise_frac=0.0)
    b = synth.generate(wl, smear=False, record_truth=True)
    res = {}
    for nm, w in (("map", wl), ("uniform", dataclasses.replace(wl, field_z2=0.0, field_r2=0.0))):
        g = oracle.Geometry(w)
        err = []
        for t in range(200):
            for k in range(b.track_nhits[t] - 1):
                out = oracle.propagate(g, b.truth_out[t, k], None, int(b.track_surf[t, k + 1]))
                assert out is not None
                err.append(np.abs(out[0][:3] - b.truth_in[t, k + 1][:3]).max())
        res[nm] = np.array(err)
    assert len(res["map"]) > 1000
    assert np.quantile(res["map"], 0.99) < 1e-3 and res["map"].max() < 5e-3
    assert np.quantile(res["uniform"], 0.99) > 3e-3


def test_zero_noise_fit_in_the_field_map():
    """Exact hits, no scattering: the fit with the field map returns the generator's state after
    the last hit within a fraction of its error; the same fit in a uniform field is many sigma off
    in curvature and direction."""
    wl = synth.workload("field", n_events=1, tracks_lo=3000, tracks_hi=3000, ms_on=False, noise_frac=0.0)
    b = synth.generate(wl, smear=False, record_truth=True)
    idx = b.track_nhits - 1
    truth = b.truth_out[np.arange(len(idx)), idx]
    pulls = {}
    for nm, w in (("map", wl), ("uniform", dataclasses.replace(wl, field_z2=0.0, field_r2=0.0))):
        r = oracle.fit(oracle.Geometry(w), b.hits, b.hit_surface, b.track_hits)
        assert np.all(r["status"] == 0)
        sig = np.sqrt(np.diagonal(oracle.unpack_cov(r["cov"]), axis1=1, axis2=2))
        d = r["p"] - truth
        d[:, 4] = _wrap(d[:, 4])
        pulls[nm] = np.abs(d[:, 3:] / sig[:, 3:])  # kappa, phi, theta
    assert pulls["map"].max() < 0.5
    assert np.quantile(pulls["uniform"][:, 0], 0.99) > 3.0 and np.quantile(pulls["uniform"][:, 1], 0.99) > 3.0


def test_pulls_in_the_field_map_with_scattering():
    """Smeared hits and scattering: pulls of kappa, phi and theta have mean 0 and width 1 with the
    field map, while a uniform-field fit widens the kappa pull."""
    wl = synth.workload("field", n_events=4, tracks_lo=3000, tracks_hi=3000, noise_frac=0.0)
    b = synth.generate(wl, record_truth=True)
    idx = b.track_nhits - 1
    truth = b.truth_out[np.arange(len(idx)), idx]
    width = {}
    for nm, w in (("map", wl), ("uniform", dataclasses.replace(wl, field_z2=0.0, field_r2=0.0))):
        r = oracle.fit(oracle.Geometry(w), b.hits, b.hit_surface, b.track_hits)
        ok = r["status"] == 0
        assert ok.mean() > 0.999
        C = oracle.unpack_cov(r["cov"])
        d = r["p"] - truth
        d[:, 4] = _wrap(d[:, 4])
        width[nm] = []
        for i in (3, 4, 5):
            pull = (d[:, i] / np.sqrt(C[:, i, i]))[ok]
            width[nm].append(pull.std())
            if nm == "map":
                assert abs(pull.mean()) < 0.05, (i, pull.mean())
                assert abs(pull.std() - 1.0) < 0.04, (i, pull.std())
    assert width["uniform"][0] > 1.15


def test_seed_curvature_uses_the_field_at_its_first_hit():
    """The seed circle is the same in any field; its kappa is the circle's curvature over k Bz at
    the seed's first hit, so the map's and the uniform field's seeds differ by bz / Bz(hit 1)."""
    wl = synth.workload("field", n_events=1, tracks_lo=200, tracks_hi=200)
    b = synth.generate(wl)
    g = oracle.Geometry(wl)
    g0 = oracle.Geometry(dataclasses.replace(wl, field_z2=0.0, field_r2=0.0))
    sh, _ = b.seeds()
    n = 0
    for ids in sh[:100]:
        a, c = oracle.seed(g, b.hits, b.hit_surface, ids), oracle.seed(g0, b.hits, b.hit_surface, ids)
        if a is None:
            continue
        pa, pc = a[0], c[0]
        assert np.array_equal(np.delete(pa, 3), np.delete(pc, 3))
        ratio = float(np.float32(wl.bz)) / _field(wl, *pa[:3])
        assert abs(pa[3] / pc[3] - ratio) < 1e-12 and abs(ratio - 1.0) > 1e-5
        n += 1
    assert n >= 90
