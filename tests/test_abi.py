"""The C-ABI library loads and exports every symbol its header declares; host-side argument
checks reject bad input before any launch (CPU only, no compute calls)."""
import ctypes
import os
import re

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include"))) if h.endswith(".h")]


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as k
    return k


def _declared():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(kf_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_api():
    names = _declared()
    for n in ("kf_build_hit_index", "kf_fit_tracks", "kf_find_tracks", "kf_find_workspace_size", "kf_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(kf):
    lib = ctypes.CDLL(kf.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(kf):
    lib = kf.load_library()
    wl = synth.workload("find")
    g = kf.Geometry(wl)
    assert g.n_bins == 64 * 32
    assert lib.kf_status_string(kf.KF_ERR_CAPACITY) == b"size above a compiled capacity"
    # bad geometry: n_surf = 0
    bad = kf.KfGeometry(3.8, 0, None, 0.01, 0.1, (ctypes.c_float * 5)(*wl.prior))
    assert lib.kf_index_bins(ctypes.byref(bad)) == kf.KF_ERR_ARG
    idx = kf.KfHitIndex(1, g.n_bins, None, None, None, None)
    rc = lib.kf_build_hit_index(ctypes.byref(bad), None, None, 1, 10, ctypes.byref(idx), None, None)
    assert rc == kf.KF_ERR_ARG
    # slab above the compiled capacity: rejected before any launch
    rc = lib.kf_build_hit_index(g.ref, ctypes.c_void_p(16), ctypes.c_void_p(16), 1, kf.KF_MAX_SLAB_HITS + 1,
                                ctypes.byref(idx), None, None)
    assert rc == kf.KF_ERR_CAPACITY
    # fit: lmax above the limit
    rc = lib.kf_fit_tracks(g.ref, None, None, None, 10, kf.KF_MAX_LMAX + 1, None, None, None, None, None, 0, None)
    assert rc == kf.KF_ERR_ARG
    # finder parameters: k above the compiled maximum
    p = kf.find_params(30.0, kf.KF_MAX_K + 1, 1, 17)
    assert lib.kf_find_workspace_size(100, ctypes.byref(p)) == 0
    # adaptive capacity: plain finding only, within [0, KF_MAX_K]
    p = kf.find_params(30.0, 8, 1, 17, adaptive_capacity=-1)
    assert lib.kf_find_workspace_size(100, ctypes.byref(p)) == 0
    p = kf.find_params(30.0, 8, 1, 17, adaptive_capacity=kf.KF_MAX_K + 1)
    assert lib.kf_find_workspace_size(100, ctypes.byref(p)) == 0
    # the allocation-free entry point has no room for adaptive capacity's overflow list
    p = kf.find_params(30.0, 8, 1, 17, adaptive_capacity=4)
    idx = kf.KfHitIndex(1, g.n_bins, None, None, None, None)
    v = ctypes.c_void_p
    rc = lib.kf_find_tracks_static(g.ref, ctypes.byref(idx), v(256), v(256), v(256), v(256), 10, ctypes.byref(p),
                                   v(256), v(256), v(256), v(256), v(256), v(256), None)
    assert rc == kf.KF_ERR_ARG
    # network kernels read feature rows as float pairs: an odd float offset is rejected
    v = ctypes.c_void_p
    assert lib.kf_mlp_forward(v(256), v(260), 1, v(512), None) == kf.KF_ERR_ARG
    assert lib.kf_mlp_loss_grad(v(256), v(260), v(1024), 1, v(512), v(768), None) == kf.KF_ERR_ARG
    # bounded-wait probe: limits outside [1 us, 1 s] and a null output are rejected
    assert lib.kf_wait_probe(0, v(256), None) == kf.KF_ERR_ARG
    assert lib.kf_wait_probe(2_000_000, v(256), None) == kf.KF_ERR_ARG
    assert lib.kf_wait_probe(1000, None, None) == kf.KF_ERR_ARG


def test_missing_library_fails_loudly(tmp_path):
    import paper_1906_02253_gb300 as k
    saved = k._lib
    try:
        k._lib = None
        with pytest.raises(k.KfError):
            k.load_library(str(tmp_path / "nope.so"))
    finally:
        k._lib = saved
