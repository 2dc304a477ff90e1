"""Pins of the oracle's helix propagation and covariance transport (CPU only).

The propagator is checked against things other than itself: the generator's independent
root-finding crossing solver (a different helix parametrisation), central finite differences
for the Jacobian, the straight-line limit, geometric invariants of the helix, and a hand-worked
Highland value with the deflection geometry for the scattering noise.
"""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import synth


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


@pytest.mark.parametrize("wl_name", ["fit_small", "hi_occ"])
def test_propagation_reproduces_generator_crossings(wl_name):
    """No smearing, no scattering: from the true state at crossing k, the oracle's closed-form
    propagation lands on the generator's root-found crossing k+1 to 1e-9 cm."""
    wl = synth.workload(wl_name, n_events=1, tracks_lo=300, tracks_hi=300, ms_on=False)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, smear=False, record_truth=True)
    worst_pos, worst_ang, n_checked = 0.0, 0.0, 0
    for t in range(b.n_tracks):
        nh = b.track_nhits[t]
        for k in range(nh - 1):
            r = oracle.propagate(g, b.truth_in[t, k], None, b.track_surf[t, k + 1])
            assert r is not None
            p, _, _, _ = r
            ref = b.truth_in[t, k + 1]
            worst_pos = max(worst_pos, np.abs(p[:3] - ref[:3]).max())
            worst_ang = max(worst_ang, abs(_wrap(p[4] - ref[4])), abs(p[5] - ref[5]), abs(p[3] - ref[3]))
            n_checked += 1
    assert n_checked > 2000
    assert worst_pos < 1e-9
    assert worst_ang < 1e-11


def _central(g, p0, surf, j, h):
    dp = np.zeros(6)
    dp[j] = h
    a = oracle.propagate(g, p0 + dp, None, surf)[0]
    b = oracle.propagate(g, p0 - dp, None, surf)[0]
    d = a - b
    d[4] = _wrap(d[4])
    return d / (2 * h)


def _fd_jacobian(g, p0, surf, h):
    """Central differences with one Richardson step (truncation error O(h^4))."""
    J = np.empty((6, 6))
    for j in range(6):
        J[:, j] = (4 * _central(g, p0, surf, j, h[j] / 2) - _central(g, p0, surf, j, h[j])) / 3
    return J


@pytest.mark.parametrize("wl_name", ["fit_batched", "hi_occ"])
def test_jacobian_matches_central_differences(wl_name):
    """The analytic, surface-projected Jacobian equals central finite differences of the full
    propagate-to-surface map (path length re-solved for every perturbation)."""
    wl = synth.workload(wl_name, n_events=1, tracks_lo=60, tracks_hi=60, ms_on=False)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, smear=False, record_truth=True)
    rng = np.random.default_rng(7)
    checked = 0
    for t in range(b.n_tracks):
        nh = b.track_nhits[t]
        k = rng.integers(0, nh - 1)
        p0 = b.truth_in[t, k].copy()
        surf = b.track_surf[t, k + 1]
        J = oracle.propagate(g, p0, None, surf)[2]
        h = np.array([1e-3, 1e-3, 1e-3, 1e-4, 1e-5, 1e-5])
        Jfd = _fd_jacobian(g, p0, surf, h)
        scale = np.maximum(np.abs(J), 1e-2)
        assert np.all(np.abs(J - Jfd) / scale < 1e-6), (t, k, J, Jfd)
        checked += 1
    assert checked == b.n_tracks


def _surface_gradient(wl, surf, p):
    s = wl.surfaces[surf]
    g = np.zeros(6)
    if s.type == synth.BARREL:
        g[0], g[1] = p[0], p[1]
    else:
        g[2] = 1.0
    return g


def test_transported_covariance_stays_on_tangent_space():
    """C' = J C J^T + Q is symmetric, annihilates the surface normal (C n = 0) and is positive
    definite on the 5D tangent space."""
    wl = synth.workload("hi_occ", n_events=1, tracks_lo=80, tracks_hi=80)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, record_truth=True)
    rng = np.random.default_rng(3)
    for t in range(b.n_tracks):
        nh = b.track_nhits[t]
        k = rng.integers(0, nh - 1)
        A = rng.normal(size=(6, 6))
        C0 = A @ A.T * 1e-3 + np.diag([1e-4, 1e-4, 1e-2, 1e-3, 1e-5, 1e-5])
        p, C, J, s = oracle.propagate(g, b.truth_out[t, k], C0, b.track_surf[t, k + 1])
        assert np.allclose(C, C.T, rtol=0, atol=1e-15 * np.abs(C).max())
        n = _surface_gradient(wl, b.track_surf[t, k + 1], p)
        n /= np.linalg.norm(n)
        assert np.linalg.norm(C @ n) <= 1e-12 * np.linalg.norm(C)
        # basis of the tangent space: orthogonal complement of n
        q, _ = np.linalg.qr(np.column_stack([n, np.eye(6)]))
        T = q[:, 1:6]
        ev = np.linalg.eigvalsh(T.T @ C @ T)
        assert ev.min() > 0


def test_straight_line_limit():
    """kappa -> 0: the crossing is the straight-line intersection with the cylinder."""
    wl = synth.workload("fit_small")
    g = oracle.Geometry(wl)
    rng = np.random.default_rng(11)
    for _ in range(200):
        phi = rng.uniform(-np.pi, np.pi)
        th = rng.uniform(0.6, 2.5)
        p0 = np.array([rng.normal() * 0.5, rng.normal() * 0.5, rng.normal(), 1e-12, phi, th])
        R = 20.0
        p = oracle.propagate(g, p0, None, 4)[0]  # layer at r = 20
        a = p0[0] * np.cos(phi) + p0[1] * np.sin(phi)
        s = -a + np.sqrt(a * a + R * R - p0[0] ** 2 - p0[1] ** 2)
        ref = np.array([p0[0] + s * np.cos(phi), p0[1] + s * np.sin(phi), p0[2] + s / np.tan(th)])
        assert np.abs(p[:3] - ref).max() < 1e-9


def test_helix_invariants():
    """Crossing lies on the cylinder, on the helix's transverse circle (radius 1/|omega|), with
    phi advanced by omega*s and z by s*cot(theta)."""
    wl = synth.workload("fit_batched")
    g = oracle.Geometry(wl)
    rng = np.random.default_rng(5)
    for _ in range(300):
        kap = rng.choice([-1, 1]) * rng.uniform(0.1, 2.0)
        p0 = np.array([4 * np.cos(0.3), 4 * np.sin(0.3), rng.normal(), kap, rng.uniform(-np.pi, np.pi),
                       rng.uniform(0.8, 2.3)])
        if np.cos(p0[4] - 0.3) < 0.3:  # moving outward
            continue
        surf = int(rng.integers(1, 17))
        r = oracle.propagate(g, p0, None, surf)
        if r is None:
            continue
        p, _, _, s = r
        R = wl.surfaces[surf].r_or_z
        w = -oracle.K_CURV * float(np.float32(wl.bz)) * kap  # geometry values are FP32
        assert abs(np.hypot(p[0], p[1]) - R) < 1e-9
        c0 = np.array([p0[0] - np.sin(p0[4]) / w, p0[1] + np.cos(p0[4]) / w])
        assert abs(np.hypot(p[0] - c0[0], p[1] - c0[1]) - 1 / abs(w)) < 1e-8
        assert abs(_wrap(p[4] - p0[4] - w * s)) < 1e-12
        assert abs(p[2] - p0[2] - s / np.tan(p0[5])) < 1e-9
        assert s > 0


def test_next_surface_rule_follows_generator_paths():
    """Without scattering, the finder's next-surface rule (next barrel layer outward vs next disk in
    the direction of motion, nearer accepted one, at most half a turn) reproduces the surface
    sequence the generator finds by searching every surface, and ends where the generator ends."""
    wl = synth.workload("hi_occ", n_events=1, tracks_lo=600, tracks_hi=600, ms_on=False)
    g = oracle.Geometry(wl)
    b = synth.generate(wl, smear=False, record_truth=True)
    n_checked = 0
    for t in range(b.n_tracks):
        nh = b.track_nhits[t]
        for k in range(nh):
            nxt, _ = oracle.next_surface(g, b.truth_in[t, k])
            want = b.track_surf[t, k + 1] if k + 1 < nh else -1
            assert nxt == want, (t, k, nxt, want)
            n_checked += 1
    assert n_checked > 5000


def _scatter_cov(x_over_x0, p0, surf, wl_name="hi_occ"):
    """Covariance after propagating a zero covariance to ``surf`` in a near-zero field (straight
    tracks from the origin), with every surface's x/X0 set to ``x_over_x0``: the scattering noise."""
    base = synth.workload(wl_name)
    surfs = [replace(s, x_over_x0=float(x_over_x0)) for s in base.surfaces]
    wl = synth.workload(wl_name, bz=1e-6, ms_on=True, surfaces=surfs)
    r = oracle.propagate(oracle.Geometry(wl), p0, None, surf)
    assert r is not None
    return r[1]


def _kick_jacobian(kap, phi, th):
    """d(kappa, phi, theta) / d(deflection) for the two deflections perpendicular to the
    direction (in the theta plane and across it), by central differences of a rotated direction
    at fixed |p| and charge; kappa = q / (p sin theta)."""
    q_over_p = kap * np.sin(th)
    u = np.array([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)])
    e1 = np.array([np.cos(th) * np.cos(phi), np.cos(th) * np.sin(phi), -np.sin(th)])
    e2 = np.array([-np.sin(phi), np.cos(phi), 0.0])
    G = np.zeros((3, 2))
    eps = 1e-6
    for j, e in enumerate((e1, e2)):
        cols = []
        for sgn in (1.0, -1.0):
            v = u + sgn * eps * e
            v /= np.linalg.norm(v)
            t = np.arccos(v[2])
            cols.append(np.array([q_over_p / np.sin(t), np.arctan2(v[1], v[0]), t]))
        d = cols[0] - cols[1]
        d[1] = _wrap(d[1])
        G[:, j] = d / (2 * eps)
    return G


def test_multiple_scattering_noise_follows_highland_and_the_deflection_geometry():
    """Sec. 3.1 multiple scattering (Highland formula, beta = 1, PDG): a 1 GeV track crossing
    2% X0 at normal incidence gets theta0 = 1.6374e-3 rad (worked out by hand: 13.6 MeV / 1 GeV x
    sqrt(0.02) x (1 + 0.038 ln 0.02)); theta0^2 scales as 1/p^2; an oblique crossing equals a
    normal one through x/X0 divided by |cos a| (the path in the layer), on barrels and disks; and
    the noise on (kappa, phi, theta) is theta0^2 G G^T with G the deflection Jacobian taken from a
    rotated direction vector."""
    x0 = np.float32(0.02)
    p_norm = np.array([0.0, 0.0, 0.0, 1.0, 0.3, np.pi / 2])  # kappa = 1 / (p sin theta): p = 1 GeV
    C = _scatter_cov(x0, p_norm, 4)
    theta0 = 1.6374e-3
    assert abs(np.sqrt(C[5, 5]) / theta0 - 1) < 1e-4
    assert abs(C[4, 4] / C[5, 5] - 1) < 1e-9
    assert abs(C[3, 3]) < 1e-15 and abs(C[3, 5]) < 1e-15
    assert np.abs(C[:3, :]).max() == 0.0

    p_two = p_norm.copy()
    p_two[3] = 0.5  # p = 2 GeV
    assert abs(_scatter_cov(x0, p_two, 4)[5, 5] * 4 / C[5, 5] - 1) < 1e-9

    for th, surf, cos_a in ((1.0, 4, np.sin(1.0)), (0.3, 17, np.cos(0.3)), (2.7, 26, np.cos(2.7))):
        kap = -1.0 / np.sin(th)  # p = 1 GeV, negative charge
        p_obl = np.array([0.0, 0.0, 0.0, kap, -2.0, th])
        C_obl = _scatter_cov(x0, p_obl, surf)
        v_ref = _scatter_cov(np.float32(x0 / abs(cos_a)), p_norm, 4)[5, 5]
        assert abs(C_obl[5, 5] / v_ref - 1) < 1e-6, (th, surf)
        G = _kick_jacobian(kap, -2.0, th)
        Q = C_obl[3:, 3:]
        assert np.abs(Q - C_obl[5, 5] * G @ G.T).max() < 1e-8 * np.abs(Q).max()
