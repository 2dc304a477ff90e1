"""The usage example of the README runs as written and gives the oracle's tracks."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_readme_example():
    import __graft_entry__ as ge
    ge.build_library()
    import synth, paper_1906_02253_gb300 as kf
    wl = synth.workload("find", n_events=2)
    batch = synth.generate(wl)
    geom = kf.Geometry(wl)
    dev = kf.to_device_event_batch(batch)
    index = kf.build_hit_index(geom, dev["hits"], dev["slab_offsets"], batch.n_events, dev["max_slab_hits"])
    params = kf.find_params(wl.chi2_cut, wl.k_max, wl.max_miss, wl.lmax)
    found = kf.find_tracks(geom, index, dev["hits"], dev["hit_surface"], dev["seed_hits"], dev["seed_event"], params)
    fitted = kf.fit_tracks(geom, dev["hits"], dev["hit_surface"], found["hits"])
    sh, st = batch.seeds()
    r = oracle.find(oracle.Geometry(wl), batch, sh, batch.track_event[st])
    assert ((found["hits"].cpu().numpy().T == r["hits"]).all(axis=1)).mean() >= 0.999
    assert (fitted["status"].cpu().numpy() == 0).mean() > 0.95
