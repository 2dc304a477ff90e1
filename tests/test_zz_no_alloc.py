"""The allocation-free finder entry point (kf_find_tracks_static) gives the results of
kf_find_tracks.

kf_find_tracks_static serves callers that cannot allocate device memory while they process
events (an online trigger process that reserves its GPU memory at start-up, a plug-in inside a
framework that owns the memory pool): its scratch is a fixed array inside the library instead of a
caller's workspace. Two calls in a row, on different events, are compared with kf_find_tracks on
the same inputs; the second call must not see anything the first left in the shared array. The
file is collected last so that a failure here stops a run only after every other test ran.
"""
import ctypes
import os

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    import __graft_entry__ as ge
    ge.build_library()
    import paper_1906_02253_gb300 as k
    lib = k.load_library()
    P = ctypes.c_void_p
    lib.kf_find_tracks_static.restype = ctypes.c_int
    lib.kf_find_tracks_static.argtypes = [ctypes.POINTER(k.KfGeometry), ctypes.POINTER(k.KfHitIndex), P, P, P, P,
                                          ctypes.c_int, ctypes.POINTER(k.KfFindParams), P, P, P, P, P, P, P]
    return k


def _outputs(n, lmax):
    return dict(hits=torch.full((lmax, n), -7, dtype=torch.int32, device="cuda"),
                nhits=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
                chi2=torch.full((n,), -7.0, dtype=torch.float32, device="cuda"),
                state=torch.full((6, n), -7.0, dtype=torch.float32, device="cuda"),
                cov=torch.full((21, n), -7.0, dtype=torch.float32, device="cuda"),
                status=torch.full((n,), -7, dtype=torch.int32, device="cuda"))


def _static_call(kf, g, idx, dev, prm, out):
    p = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    n = dev["seed_hits"].shape[1]
    return kf.load_library().kf_find_tracks_static(
        g.ref, ctypes.byref(idx.c), p(dev["hits"]), p(dev["hit_surface"]), p(dev["seed_hits"]), p(dev["seed_event"]),
        n, ctypes.byref(prm), p(out["hits"]), p(out["nhits"]), p(out["chi2"]), p(out["state"]), p(out["cov"]),
        p(out["status"]), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.mark.parametrize("first,second", [(("find", 31), ("find", 32)), (("hi_occ", 33), ("find", 34))])
def test_static_entry_point_matches_workspace_entry_point(kf, first, second):
    for name, seed in (first, second):
        wl = synth.workload(name, n_events=2, tracks_lo=1000, tracks_hi=2500, seed=seed)
        b = synth.generate(wl)
        g = kf.Geometry(wl)
        dev = kf.to_device_event_batch(b)
        idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
        prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
        ref = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
        out = _outputs(dev["seed_hits"].shape[1], wl.lmax)
        assert _static_call(kf, g, idx, dev, prm, out) == kf.KF_OK
        torch.cuda.synchronize()
        for k in ("hits", "nhits", "status"):
            assert torch.equal(out[k], ref[k]), k
        ok = ref["status"] == 0
        # the same kernels run on the same inputs; the parity tolerances bound any difference
        assert torch.allclose(out["chi2"][ok], ref["chi2"][ok], rtol=1e-3, atol=0)
        assert torch.allclose(out["state"][:, ok], ref["state"][:, ok], rtol=1e-4, atol=1e-6)
        assert torch.allclose(out["cov"][:, ok], ref["cov"][:, ok], rtol=1e-3, atol=1e-9)


def _compare(out, ref):
    for k in ("hits", "nhits", "status"):
        assert torch.equal(out[k], ref[k]), k
    ok = ref["status"] == 0
    assert torch.allclose(out["chi2"][ok], ref["chi2"][ok], rtol=1e-3, atol=0)
    assert torch.allclose(out["state"][:, ok], ref["state"][:, ok], rtol=1e-4, atol=1e-6)
    assert torch.allclose(out["cov"][:, ok], ref["cov"][:, ok], rtol=1e-3, atol=1e-9)


def test_static_entry_point_learned_proposal_between_plain_calls(kf):
    """The learned proposal keeps its weight fragments in the array, after the seed
    states: plain, learned (top_n rule, score margin, window ranking with a margin), plain again on
    the same events must each match kf_find_tracks."""
    z = np.load(os.path.join(os.path.dirname(kf.__file__), "data", "mlp_learned.npz"))
    buf = kf.mlp_buffer(z["weights"], z["mean"], z["sd"], device="cuda")
    wl = synth.workload("learned", n_events=2, tracks_lo=1500, tracks_hi=3000, seed=35)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    for mlp, top_n, margin, window in ((None, 0, 0.0, False), (buf, 2, 0.0, False), (None, 0, 0.0, False),
                                       (buf, 1, 0.0, False), (buf, 2, 0.7, False), (buf, 2, 0.7, True)):
        prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax, mlp=mlp, top_n=top_n, score_margin=margin,
                             window_ranking=window)
        ref = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
        out = _outputs(dev["seed_hits"].shape[1], wl.lmax)
        assert _static_call(kf, g, idx, dev, prm, out) == kf.KF_OK
        torch.cuda.synchronize()
        _compare(out, ref)


def test_static_entry_point_at_its_seed_capacity(kf):
    """Exactly KF_STATIC_MAX_SEEDS seeds (the largest call the array serves)."""
    wl = synth.workload("find", n_events=14, seed=36)
    b = synth.generate(wl)
    g = kf.Geometry(wl)
    dev = kf.to_device_event_batch(b)
    n = 65536
    assert dev["seed_hits"].shape[1] >= n
    dev["seed_hits"] = dev["seed_hits"][:, :n].contiguous()
    dev["seed_event"] = dev["seed_event"][:n].contiguous()
    idx = kf.build_hit_index(g, dev["hits"], dev["slab_offsets"], b.n_events, dev["max_slab_hits"])
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
    ref = kf.find_tracks(g, idx, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], prm)
    out = _outputs(n, wl.lmax)
    assert _static_call(kf, g, idx, dev, prm, out) == kf.KF_OK
    torch.cuda.synchronize()
    _compare(out, ref)


def test_static_entry_point_rejects_too_many_seeds(kf):
    wl = synth.workload("find")
    g = kf.Geometry(wl)
    idx = kf.KfHitIndex(1, g.n_bins, None, None, None, None)
    prm = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
    rc = kf.load_library().kf_find_tracks_static(g.ref, ctypes.byref(idx), None, None, None, None,
                                                 65536 + 1, ctypes.byref(prm), None, None, None, None, None,
                                                 None, None)
    assert rc == kf.KF_ERR_CAPACITY
