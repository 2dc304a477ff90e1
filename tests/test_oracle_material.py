"""Pins of the oracle's material map and mean energy loss (Sec. 3.1 reading: material indexed in
r-z, energy loss in the layers), CPU only.

The generator applies the same physics with its own code on the exact crossings (a different
helix parametrisation and root finder), so zero-noise tracks test the oracle's mean loss and its
material interpolation; pulls test the covariance; finite differences test the kappa scaling.
"""
import dataclasses

import numpy as np

import oracle
import synth


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _last(batch, arr):
    idx = batch.track_nhits - 1
    return arr[np.arange(len(idx)), idx]


def test_material_map_and_energy_loss_of_exact_tracks_are_reproduced():
    """No scattering, exact hits, material map + energy loss: the fit returns the generator's state
    after the last layer's loss; without the loss in the fit, kappa is off by many sigma."""
    wl = synth.workload("material", n_events=1, tracks_lo=800, tracks_hi=800, ms_on=False)
    b = synth.generate(wl, smear=False, record_truth=True)
    r = oracle.fit(oracle.Geometry(wl), b.hits, b.hit_surface, b.track_hits)
    assert np.all(r["status"] == 0)
    truth = _last(b, b.truth_out)
    sig = np.sqrt(np.diagonal(oracle.unpack_cov(r["cov"]), axis1=1, axis2=2))
    d = r["p"] - truth
    d[:, 4] = _wrap(d[:, 4])
    assert np.abs(d[:, 3] / sig[:, 3]).max() < 2e-3
    assert np.abs(d[:, 5] / sig[:, 5]).max() < 2e-3
    assert r["chi2"].max() < 1e-4
    # the same fit without the loss: the seed's curvature is that of the first layers and the
    # later layers are fitted with the wrong momentum
    r0 = oracle.fit(oracle.Geometry(dataclasses.replace(wl, eloss=0.0)), b.hits, b.hit_surface, b.track_hits)
    d0 = np.abs(r0["p"][:, 3] - truth[:, 3]) / sig[:, 3]
    assert np.quantile(d0, 0.9) > 1.0 and d0.max() > 10.0  # low-momentum tracks lose most
    assert np.median(r0["chi2"]) > 100 * max(np.median(r["chi2"]), 1e-12)


def test_pulls_with_material_map_and_energy_loss():
    """Scattering with the material map and energy loss: parameter pulls have mean 0 and width 1
    and chi2/ndof is 1; a fit that ignores the loss biases kappa."""
    wl = synth.workload("material", n_events=4, tracks_lo=3000, tracks_hi=3000)
    b = synth.generate(wl, record_truth=True)
    r = oracle.fit(oracle.Geometry(wl), b.hits, b.hit_surface, b.track_hits)
    assert np.all(r["status"] == 0)
    truth = _last(b, b.truth_out)
    C = oracle.unpack_cov(r["cov"])
    d = r["p"] - truth
    d[:, 4] = _wrap(d[:, 4])
    for i in (2, 3, 4, 5):
        pull = d[:, i] / np.sqrt(C[:, i, i])
        assert abs(pull.mean()) < 0.05, (i, pull.mean())
        assert abs(pull.std() - 1.0) < 0.04, (i, pull.std())
    assert abs(r["chi2"].sum() / r["ndof"].sum() - 1.0) < 0.02
    r0 = oracle.fit(oracle.Geometry(dataclasses.replace(wl, eloss=0.0)), b.hits, b.hit_surface, b.track_hits)
    pull0 = (r0["p"][:, 3] - truth[:, 3]) / np.sqrt(oracle.unpack_cov(r0["cov"])[:, 3, 3])
    q = np.sign(truth[:, 3])
    assert abs((pull0 * q).mean()) > 0.1  # |kappa| too small without the loss (0.009 standard error)


def test_energy_loss_kappa_factor_matches_finite_differences():
    """d kappa'/d kappa of the propagation with energy loss (no scattering) equals the factor the
    covariance transport applies to kappa's row and column."""
    wl = synth.workload("material", n_events=1, tracks_lo=20, tracks_hi=20, ms_on=False)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, smear=False, record_truth=True)
    rng = np.random.default_rng(7)
    checked = 0
    for t in rng.choice(b.n_tracks, 10, replace=False):
        p0 = b.truth_out[t, 0].copy()
        surf = int(b.track_surf[t, 1])
        Ck = np.zeros((6, 6))
        Ck[3, 3] = 1.0
        out = oracle.propagate(g, p0, Ck, surf)
        if out is None:
            continue
        h = 1e-4 * abs(p0[3])
        kp = []
        for sgn in (+1, -1):
            q = p0.copy()
            q[3] += sgn * h
            kp.append(oracle.propagate(g, q, None, surf)[0][3])
        fd = (kp[0] - kp[1]) / (2 * h)
        assert abs(np.sqrt(out[1][3, 3]) - abs(fd)) < 1e-5 * abs(fd), (t, fd, out[1][3, 3])
        assert abs(fd) > 1.0  # kappa grows: the loss is active
        checked += 1
    assert checked >= 5


def test_material_map_interpolation_closed_form():
    """One barrel crossing without scattering at a chosen z: the loss uses x/X0 interpolated
    linearly between the two map nodes around z (and not the surface's nominal x_over_x0)."""
    wl = synth.workload("material", ms_on=False)
    g = oracle.Geometry(wl)
    s = wl.surfaces[5]
    nodes = np.asarray(wl.material[5], np.float32).astype(np.float64)
    # a stiff track from the previous layer towards z = zc on layer 5, crossing nearly radially
    zc = s.lo + (s.hi - s.lo) * 2.4 / 7
    r_prev = wl.surfaces[4].r_or_z
    theta = np.arctan2(s.r_or_z - r_prev, zc * (1 - r_prev / s.r_or_z))
    p0 = np.array([r_prev, 0.0, zc * r_prev / s.r_or_z, 1e-6, 0.0, theta])
    out = oracle.propagate(g, p0, None, 5)
    assert out is not None
    pe = out[0]
    u = (pe[2] - s.lo) / (s.hi - s.lo) * 7
    k = int(np.floor(u))
    xx0 = nodes[k] + (u - k) * (nodes[k + 1] - nodes[k])
    cos_a = np.sin(theta)  # radial crossing: the angle to the normal is the dip
    p = 1.0 / (1e-6 * np.sin(theta))
    m = np.float32(wl.mass)
    e1 = np.sqrt(p * p + m * m) - np.float32(wl.eloss) * xx0 / cos_a
    p1 = np.sqrt(e1 * e1 - m * m)
    assert abs(pe[3] / 1e-6 - p / p1) < 1e-9
    assert abs(xx0 - s.x_over_x0) > 0.2 * s.x_over_x0  # the map differs from the nominal value here
