"""Accuracy of the hand-written trigonometry on the Kalman path, on the GPU through kf_math_probe
(the same code and compiler flags as the finder and the fit).

sincos_small (Cody-Waite reduction and Taylor series), the small-angle arctangent series of the
residual angles and the half-angle helix functions replace sincosf/atan2f on the hot path. Each is
compared over dense grids of the arguments the path gives it with the FP64 value of the same FP32
argument, in units of the FP32 spacing (ulp) at the exact value, and with CUDA's own FP32
functions (torch.sin, torch.cos, torch.atan on the device, which are within 2 ulp of the exact
value themselves). Bounds: 2 ulp for sin and cos, 4 ulp where a fast-math division enters (the
arctangent's a / b and the half-angle q = sin(h) / h beyond the series range).
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as k
    k.load_library()
    return k


def _ulps(got, exact):
    """|got - exact| in units of the FP32 spacing at |exact| (normal range)."""
    got = np.asarray(got, np.float64)
    sp = np.spacing(np.maximum(np.abs(exact), 1e-37).astype(np.float32)).astype(np.float64)
    return np.abs(got - exact) / sp


def _grid(rng, lo, hi, n):
    x = np.concatenate([np.linspace(lo, hi, n // 2), rng.uniform(lo, hi, n - n // 2)]).astype(np.float32)
    return x[np.abs(x) > 1e-30]


def test_sincos_small_accuracy(kf):
    rng = np.random.default_rng(5)
    parts = [_grid(rng, -np.pi, np.pi, 1 << 20), _grid(rng, -100.0, 100.0, 1 << 20)]
    # arguments next to multiples of pi/2, where the reduction decides everything
    k = np.arange(-60, 61)
    near = (k[:, None] * (np.pi / 2) + np.linspace(-1e-3, 1e-3, 401)[None, :]).ravel()
    parts.append(near.astype(np.float32))
    x = np.concatenate(parts)
    xt = torch.from_numpy(x).cuda()
    s, c, _ = kf.math_probe(kf.PROBE_SINCOS, xt)
    s, c = s.cpu().numpy(), c.cpu().numpy()
    x64 = x.astype(np.float64)
    es, ec = _ulps(s, np.sin(x64)), _ulps(c, np.cos(x64))
    assert es.max() <= 2.0, (es.max(), x[es.argmax()])
    assert ec.max() <= 2.0, (ec.max(), x[ec.argmax()])
    # against CUDA's FP32 sin and cos (each within 2 ulp of the exact value)
    ls, lc = torch.sin(xt).cpu().numpy(), torch.cos(xt).cpu().numpy()
    assert _ulps(s, ls.astype(np.float64)).max() <= 4.0
    assert _ulps(c, lc.astype(np.float64)).max() <= 4.0
    # beyond the argument bound the result is NaN, never a wrong number
    big = torch.tensor([1.5e5, -3e7, float("inf")], device="cuda")
    s2, c2, _ = kf.math_probe(kf.PROBE_SINCOS, big)
    assert torch.isnan(s2).all() and torch.isnan(c2).all()


def test_atan_small_accuracy(kf):
    """Residual angles: b > 0 and |a| < 0.05 b (the window_chi2 and residual branch condition)."""
    rng = np.random.default_rng(6)
    n = 1 << 21
    b = (10.0 ** rng.uniform(-2, 3, n)).astype(np.float32)
    t = np.concatenate([np.linspace(-0.0499, 0.0499, n // 2), rng.uniform(-0.0499, 0.0499, n - n // 2)])
    a = (t * b).astype(np.float32)
    keep = (np.abs(a) < 0.05 * b) & (np.abs(a) > 1e-30)
    a, b = a[keep], b[keep]
    o, _, _ = kf.math_probe(kf.PROBE_ATAN_SMALL, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda())
    o = o.cpu().numpy()
    exact = np.arctan(a.astype(np.float64) / b.astype(np.float64))
    e = _ulps(o, exact)
    assert e.max() <= 4.0, (e.max(), a[e.argmax()], b[e.argmax()])
    lib = torch.atan2(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    assert _ulps(o, lib.astype(np.float64)).max() <= 6.0


def test_half_angle_accuracy(kf):
    """Helix step functions of D = omega s: the series branch (|D/2| < 0.1) and the sincos branch."""
    rng = np.random.default_rng(7)
    D = np.concatenate([_grid(rng, -0.2, 0.2, 1 << 20), _grid(rng, -6.0, 6.0, 1 << 20),
                        np.array([0.19999, 0.2, 0.20001, -0.2, 1e-20], np.float32)])
    q, sh, ch = (v.cpu().numpy() for v in kf.math_probe(kf.PROBE_HALF_ANGLE, torch.from_numpy(D).cuda()))
    h = 0.5 * D.astype(np.float64)
    eq = _ulps(q, np.sin(h) / h)
    es = _ulps(sh, np.sin(h))
    ec = _ulps(ch, np.cos(h))
    series = np.abs(h) < 0.1
    assert eq[series].max() <= 2.0 and es[series].max() <= 2.0 and ec[series].max() <= 2.0
    assert eq.max() <= 4.0, (eq.max(), D[eq.argmax()])
    assert es.max() <= 2.0 and ec.max() <= 2.0


def test_probe_rejects_bad_arguments(kf):
    lib = kf.load_library()
    assert lib.kf_math_probe(7, None, None, 1, None, None, None, None) == kf.KF_ERR_ARG
    assert lib.kf_math_probe(kf.PROBE_SINCOS, None, None, -1, None, None, None, None) == kf.KF_ERR_ARG
    assert lib.kf_math_probe(kf.PROBE_SINCOS, None, None, 0, None, None, None, None) == kf.KF_OK
