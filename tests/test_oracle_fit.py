"""Pins of the oracle's Kalman-filter track fit (CPU only).

Checked against: the generator's truth (zero-noise fits reproduce it), the chi-square law with
2 degrees of freedom for predicted residuals, unit-width pulls (with and without scattering,
which validates the scattering noise), an independent iterated batch least-squares fit built on
the generator's own helix model, and covariance invariants.
"""
import numpy as np
import pytest
from scipy import optimize, stats

import oracle
import synth


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _last(batch, arr):
    return arr[np.arange(batch.n_tracks), batch.track_nhits - 1]


def test_zero_noise_fit_recovers_truth():
    """Exact hits, no scattering: the seed circle is exact, every residual vanishes, and the fit
    returns the true state at the last hit. The only error left is the FP32 storage of the hits
    (half an ulp of phi ~ 1.2e-7 rad times r <= 40 cm, and of z)."""
    wl = synth.workload("fit_small")
    g = oracle.Geometry(wl)
    b = synth.generate(wl, smear=False, record_truth=True)
    r = oracle.fit(g, b.hits, b.hit_surface, b.track_hits)
    assert np.all(r["status"] == 0)
    d = r["p"] - _last(b, b.truth_in)
    d[:, 4] = _wrap(d[:, 4])
    assert np.abs(d[:, :3]).max() < 2e-5          # cm
    # In units of the fit's own uncertainty: FP32 hit rounding (~5e-6 cm) over a 0.01 cm
    # resolution leaves the estimate within a few 1e-4 sigma of the truth.
    sig = np.sqrt(np.diagonal(oracle.unpack_cov(r["cov"]), axis1=1, axis2=2))
    assert np.abs(d[:, 2:] / sig[:, 2:]).max() < 2e-3
    # chi2 of FP32 rounding alone: residuals ~1e-6 of sigma
    assert r["chi2"].max() < 1e-5
    assert np.all(r["ndof"] == 2 * 10 - 5)


@pytest.mark.parametrize("wl_name,ms", [("fit_small", False), ("fit_batched", True)])
def test_predicted_chi2_and_pulls(wl_name, ms):
    """Per-hit predicted chi2 of hits 5.. follows chi2(2); residual pulls and final-parameter pulls
    have mean 0 and width 1 (>= 10^4 tracks). With scattering on, the truth to compare with is the
    state after the last surface's kick, which the filter's noise term describes. Hit 4 is left
    out: the prior is centred on the seed made from hits 1-3, a data-dependent centre that
    narrows the predicted spread at the first hit after them (about +7% in its mean chi2)."""
    wl = synth.workload(wl_name, n_events=4, tracks_lo=3000, tracks_hi=3000, ms_on=ms)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, record_truth=True)
    r = oracle.fit(g, b.hits, b.hit_surface, b.track_hits, per_hit=True)
    assert np.all(r["status"] == 0)
    c2 = r["hit_chi2"][:, 4:].ravel()
    assert abs(c2.mean() - 2.0) < 0.03
    ks = stats.kstest(c2[::7], stats.chi2(2).cdf)
    assert ks.pvalue > 0.01, ks
    pulls = r["hit_pull"][:, 4:].reshape(-1, 2)
    assert np.all(np.abs(pulls.mean(0)) < 0.02)
    assert np.all(np.abs(pulls.std(0) - 1.0) < 0.02)
    truth = _last(b, b.truth_out)
    C = oracle.unpack_cov(r["cov"])
    d = r["p"] - truth
    d[:, 4] = _wrap(d[:, 4])
    for i in (2, 3, 4, 5):
        pull = d[:, i] / np.sqrt(C[:, i, i])
        assert abs(pull.mean()) < 0.05, (i, pull.mean())
        assert abs(pull.std() - 1.0) < 0.03, (i, pull.std())
    # total chi2 / ndof
    assert abs((r["chi2"].sum() / r["ndof"].sum()) - 1.0) < 0.02


def test_fit_covariance_invariants():
    """Final covariance: symmetric (packed storage), positive definite on the tangent space, and
    (nearly) annihilating the barrel normal. The update keeps C n = 0 for the normal at the
    predicted position; the updated position has moved tangentially by |K r| <~ 0.05 cm, which
    tilts the normal by |K r| / R, so C n_updated is bounded by 1e-3 of |C| at r >= 4 cm."""
    wl = synth.workload("fit_batched", n_events=1, tracks_lo=500, tracks_hi=500)
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    r = oracle.fit(g, b.hits, b.hit_surface, b.track_hits)
    C = oracle.unpack_cov(r["cov"])
    for t in range(b.n_tracks):
        n = np.array([r["p"][t, 0], r["p"][t, 1], 0, 0, 0, 0])
        n /= np.linalg.norm(n)
        assert np.linalg.norm(C[t] @ n) <= 1e-3 * np.linalg.norm(C[t])
        q, _ = np.linalg.qr(np.column_stack([n, np.eye(6)]))
        T = q[:, 1:6]
        assert np.linalg.eigvalsh(T.T @ C[t] @ T).min() > 0


# ---- independent batch least squares on the generator's helix model --------------------------

def _model_hits(wl, x5, R1, surfaces):
    """Track from local parameters at the first barrel layer (phi_pos, z, kappa, phi, theta):
    predicted (phi_pos, z) at every surface, propagated with the generator's crossing solver."""
    bz = float(np.float32(wl.bz))
    ph, z, kap, phi, th = x5
    pos = np.array([R1 * np.cos(ph), R1 * np.sin(ph), z])
    pt = 1.0 / abs(kap)
    q = 1 if kap > 0 else -1
    mom = np.array([pt * np.cos(phi), pt * np.sin(phi), pt / np.tan(th)])
    out = [(ph, z)]
    for s in surfaces[1:]:
        r = synth.cross(0, float(np.float32(wl.surfaces[s].r_or_z)), bz, q, pos, mom)
        assert r is not None
        pos, mom, _ = r
        out.append((np.arctan2(pos[1], pos[0]), pos[2]))
    return out, pos, mom, q


@pytest.mark.parametrize("scale,tol", [(1e-3, 1e-3), (1.0, 0.2)])
def test_kalman_equals_batch_least_squares(scale, tol):
    """Without process noise the Kalman filter is recursive least squares: the filtered state at
    the last hit equals the iterated (Gauss-Newton) batch fit of all hits plus the same prior,
    propagated to the last hit. The batch side uses only the generator's helix model.

    The filter linearises each step at its running estimate (extended Kalman filter), which is
    what the method prescribes; the gap to the iterated fit is therefore first order in the
    resolution. With resolution and prior scaled by 1e-3 and 1e-2 the two agree to 1e-3 sigma; at
    nominal resolution the linearisation at the 3-hit seed leaves up to ~0.14 sigma in theta."""
    wl = synth.workload("fit_small", n_events=1, tracks_lo=40, tracks_hi=40, sigma_rphi=0.01 * scale,
                        sigma_2nd=0.1 * scale, prior=tuple(np.array((0.1, 1.0, 0.5, 0.05, 0.05)) * min(1.0, 10 * scale)))
    g = oracle.Geometry(wl)
    b = synth.generate(wl)
    r = oracle.fit(g, b.hits, b.hit_surface, b.track_hits)
    C = oracle.unpack_cov(r["cov"])
    sr, sz = wl.sigma_rphi, wl.sigma_2nd
    pri = np.array(wl.prior)
    worst = 0.0
    for t in range(b.n_tracks):
        ids = b.track_hits[t]
        surfs = b.hit_surface[ids]
        R = np.array([float(np.float32(wl.surfaces[s].r_or_z)) for s in surfs])
        hphi = b.hits[ids, 0].astype(np.float64)
        hz = b.hits[ids, 1].astype(np.float64)
        p0, _ = oracle.seed(g, b.hits, b.hit_surface, ids[:3])
        ph0 = np.arctan2(p0[1], p0[0])
        x_seed = np.array([ph0, p0[2], p0[3], p0[4], p0[5]])
        sd_seed = np.array([pri[0] / R[0], pri[1], pri[2], pri[3], pri[4]])

        def resid(x5):
            pred, _, _, _ = _model_hits(wl, x5, R[0], surfs)
            out = []
            for k, (pp, pz) in enumerate(pred):
                out.append(R[k] * _wrap(hphi[k] - pp) / sr)
                out.append((hz[k] - pz) / sz)
            d = x5 - x_seed
            d[0] = _wrap(d[0])
            d[3] = _wrap(d[3])
            out.extend(d / sd_seed)
            return np.array(out)

        sol = optimize.least_squares(resid, x_seed, method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15)
        _, pos, mom, q = _model_hits(wl, sol.x, R[0], surfs)
        pt = np.hypot(mom[0], mom[1])
        ref = np.array([pos[0], pos[1], pos[2], q / pt, np.arctan2(mom[1], mom[0]), np.arctan2(pt, mom[2])])
        d = r["p"][t] - ref
        d[4] = _wrap(d[4])
        sig = np.sqrt(np.diag(C[t]))
        worst = max(worst, np.max(np.abs(d[2:]) / sig[2:]), np.hypot(d[0], d[1]) / np.sqrt(C[t, 0, 0] + C[t, 1, 1]))
    assert worst < tol, worst
