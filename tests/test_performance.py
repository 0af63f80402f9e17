"""Host-side tracking-performance tools (efficiency / fake rate / duplicates of the track
candidates) fed with the oracle's track candidates on generator truth. CPU only."""
import numpy as np

import oracle
from paper_2403_13166_gb300 import performance, synth, truth


def test_layer_chains_follow_the_module_map_relation():
    ch = set(truth.T5_CHAINS)
    assert {(1, 2, 3, 4, 5), (2, 3, 4, 5, 6), (7, 8, 9, 10, 11), (3, 4, 5, 6, 7), (1, 7, 8, 9, 10)} <= ch
    assert all(synth.layers_adjacent(a, 1, b, 1) for c in ch for a, b in zip(c, c[1:]))
    assert (1, 2, 3, 5, 6) not in ch and len(ch) == 21


def test_toy_muons_are_found_once_without_fakes(geom_toy, cuts):
    every = dict(cuts, wp=np.float32(0.0))
    t = performance.Tally()
    for i in range(4):
        e = synth.toy_event(geom_toy, i)
        r = oracle.run_event(geom_toy, e, every, None)
        t.add(r.tc_hits(), e, geom_toy.layer)
    res = t.result()
    assert res["findable"] > 150
    assert res["efficiency"] >= 0.97 and res["fake_rate"] <= 0.02 and res["duplicate_rate"] <= 0.05
    assert all(v is None or 0.9 <= v <= 1.0 for v in res["efficiency_vs_pt"])


def test_candidate_kinematics_match_the_generated_track(geom_toy, cuts):
    every = dict(cuts, wp=np.float32(0.0))
    e = synth.toy_event(geom_toy, 5)
    r = oracle.run_event(geom_toy, e, every, None)
    tc = r.tc_hits()
    m = truth.match_particle(tc, e.pid)
    pt, eta = performance.candidate_kinematics(tc[m >= 0], e)
    true_pt, true_eta = e.particles["pt"][m[m >= 0]], e.particles["eta"][m[m >= 0]]
    assert len(pt) > 30
    assert np.median(np.abs(pt / true_pt - 1.0)) < 0.02
    assert np.median(np.abs(eta - true_eta)) < 0.01


def test_muon_cube_sample():
    g = synth.build_geometry(True)
    e = synth.muon_cube_event(g, 0)
    P = e.particles
    assert np.all(np.abs(np.stack([P["vx"], P["vy"], P["vz"]])) <= 2.5)
    c = synth.pre_dnn_cuts(20.0)
    t = performance.Tally()
    for i in range(3):
        e = synth.muon_cube_event(g, i)
        t.add(oracle.run_event(g, e, c, None).tc_hits(), e, g.layer)
    res = t.result()
    assert res["findable"] >= 30 and res["efficiency"] > 0.8 and res["fake_rate"] < 0.05
