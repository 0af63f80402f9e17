"""Pins of the oracle's steps 1-4 against things other than itself.

* closed-form helices: curvature value and sign, pT threshold, luminous-region road,
  z linear in arc length (Section 1: "consistency with a continuous, helical trajectory",
  MDs "required to have pT > 0.8 GeV");
* brute force: module-indexed enumeration == enumeration without module indexing;
* truth: isolated muons are found with near-100% efficiency (Section 1 matching rule).
"""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import synth, truth

K = synth.K_FIELD


def _run(g, e, cuts, brute=False):
    return oracle.run_event(g, e, cuts, synth.mlp_flat(synth.xavier_mlp()), 2, brute=brute)


def _anchor(e, i):
    x, y, z = float(e.x[i]), float(e.y[i]), float(e.z[i])
    r = np.float32(np.sqrt(np.float32(x) * np.float32(x) + np.float32(y) * np.float32(y)))
    return np.array([x, y, z, r], np.float32)


def _true_layers(g, e, pid):
    """(lower index, upper index) of the particle's hit pair in each module crossed, by layer."""
    out = {}
    for m in np.unique(e.sensor[e.pid == pid] // 2):
        lo = np.nonzero((e.pid == pid) & (e.sensor == 2 * m))[0]
        up = np.nonzero((e.pid == pid) & (e.sensor == 2 * m + 1))[0]
        if lo.size and up.size:
            out.setdefault(int(g.layer[m]), []).append((int(lo[0]), int(up[0]), int(m)))
    return out


# ------------------------------------------------------------------ curvature: value and sign
@pytest.mark.parametrize("q", [-1.0, 1.0])
@pytest.mark.parametrize("pt", [0.9, 2.0, 10.0])
def test_triplet_curvature_equals_helix(geom_toy, cuts, q, pt):
    e = synth.muon_event(geom_toy, [pt], [0.3], [0.7], [q], sigma=0.0)
    r = _run(geom_toy, e, cuts)
    m = truth.match_particle(r.t3_hits(), e.pid)
    assert (m == 0).sum() >= 3
    k_true = -q * K / pt   # a clockwise (q > 0) turn gives a negative cross product
    k = r.t3_kappa[m == 0].astype(np.float64)
    assert np.all(np.abs(k - k_true) <= 2e-3 * abs(k_true))
    # MD and LS curvature estimates carry the same sign convention
    ls_m = truth.match_particle(r.ls_hits(), e.pid)
    assert np.all(np.sign(r.ls_kappa[ls_m == 0]) == np.sign(k_true))
    assert np.all(np.abs(r.ls_kappa[ls_m == 0] - k_true) < 0.05 * abs(k_true) + 1e-5)


def test_straight_line_has_zero_curvature(cuts):
    P = [np.array([r * np.cos(0.4), r * np.sin(0.4), 0.3 * r, r], np.float32) for r in (23.0, 36.0, 51.0)]
    ok, k = oracle.t3_cut(P[0], P[1], P[2], cuts)
    assert ok and abs(float(k)) < 1e-6


def test_circle_through_three_points(cuts):
    # points on a circle of radius 200 cm centred at (0, -200): curvature 1/200, and the
    # path (0,0)->(a)->(b) turns clockwise, so the signed value is -1/200
    R = 200.0
    pts = []
    for t in (0.12, 0.2, 0.29):
        x, y = R * np.sin(t), -R + R * np.cos(t)
        pts.append(np.array([x, y, 0.0, np.hypot(x, y)], np.float32))
    ok, k = oracle.t3_cut(pts[0], pts[1], pts[2], cuts)
    assert ok
    assert abs(float(k) + 1.0 / R) < 1e-4 / R


# ------------------------------------------------------------------ pT threshold (Section 1)
@pytest.mark.parametrize("q", [-1.0, 1.0])
def test_pt_threshold_whole_chain(geom_toy, cuts, q):
    phis = np.linspace(-3.0, 3.0, 7)
    # above threshold: every track yields truth-matched T5s
    hi = synth.muon_event(geom_toy, [0.8 * 1.05] * 7, [0.2] * 7, phis, [q] * 7, sigma=0.0)
    r = _run(geom_toy, hi, cuts)
    m = truth.match_particle(r.t5_hits(), hi.pid)
    assert set(m[m >= 0]) == set(range(7))
    # below threshold: no segment between two of a track's own MDs
    lo = synth.muon_event(geom_toy, [0.8 * 0.8] * 7, [0.2] * 7, phis, [q] * 7, sigma=0.0)
    r = _run(geom_toy, lo, cuts)
    assert len(truth.match_particle(r.ls_hits(), lo.pid)) == 0 or \
        (truth.match_particle(r.ls_hits(), lo.pid) < 0).all()
    assert r.counts["t5"] == 0


def test_ls_bend_threshold_exact_points(geom_toy, cuts):
    for pt, expect in ((0.8 * 1.05, True), (0.8 * 0.8, False)):
        for q in (-1.0, 1.0):
            e = synth.muon_event(geom_toy, [pt], [0.1], [1.1], [q], sigma=0.0)
            lay = _true_layers(geom_toy, e, 0)
            pairs = [l for l in (1, 2, 3, 4, 5) if l in lay and l + 1 in lay]
            assert len(pairs) >= 4
            for l in pairs:
                (lo_a, up_a, _), (lo_b, up_b, _) = lay[l][0], lay[l + 1][0]
                A, B = _anchor(e, lo_a), _anchor(e, lo_b)
                ok, _ = oracle.ls_cut(A, B, 0.0, 0.0, 0, 0, cuts)
                assert ok == expect, (pt, q, l)


# ------------------------------------------------------------------ luminous-region road
def test_luminous_region_road(geom_toy, cuts):
    inside = synth.muon_event(geom_toy, [3.0] * 4, [0.3, -0.3, 0.5, 0.0], [0.1, 1.2, 2.3, -2.0],
                              [1, -1, 1, -1], vertex=(0.0, 0.0, 15.0), sigma=0.0)
    r = _run(geom_toy, inside, cuts)
    m = truth.match_particle(r.t5_hits(), inside.pid)
    assert set(m[m >= 0]) == {0, 1, 2, 3}
    outside = synth.muon_event(geom_toy, [3.0] * 4, [0.3, -0.3, 0.5, 0.0], [0.1, 1.2, 2.3, -2.0],
                               [1, -1, 1, -1], vertex=(0.0, 0.0, 26.0), sigma=0.0)
    r = _run(geom_toy, outside, cuts)
    assert r.counts["ls"] == 0


# ------------------------------------------------------------------ z linear in arc length
def test_rz_consistency_cuts(geom_toy, cuts):
    e = synth.muon_event(geom_toy, [1.5], [0.6], [0.4], [1.0], sigma=0.0)
    lay = _true_layers(geom_toy, e, 0)
    P = [_anchor(e, lay[l][0][0]) for l in (1, 2, 3, 4, 5)]
    ok, ka = oracle.t3_cut(P[0], P[1], P[2], cuts)
    ok2, kb = oracle.t3_cut(P[2], P[3], P[4], cuts)
    assert ok and ok2
    assert oracle.t5_cut(np.stack(P), ka, kb, cuts)
    for dz, expect in ((0.01, True), (0.05, False)):
        Q = [p.copy() for p in P]
        Q[1][2] += dz
        assert oracle.t3_cut(Q[0], Q[1], Q[2], cuts)[0] == expect
        Q = [p.copy() for p in P]
        Q[3][2] += dz if expect else 0.06
        assert oracle.t5_cut(np.stack(Q), ka, kb, cuts) == expect
    # opposite-sign curvatures never form a quintuplet
    assert not oracle.t5_cut(np.stack(P), ka, -kb, cuts)


# ------------------------------------------------------------------ endcap path
def test_endcap_track_found(geom_full, cuts):
    e = synth.muon_event(geom_full, [2.0, 5.0], [2.1, -1.9], [0.5, -1.5], [1, -1], sigma=0.0)
    r = _run(geom_full, e, cuts)
    md_m = truth.match_particle(r.md_hits(), e.pid)
    ec = geom_full.subdet[r.md_mod] == 1
    assert (ec & (md_m >= 0)).sum() >= 8
    m = truth.match_particle(r.t5_hits(), e.pid)
    assert set(m[m >= 0]) == {0, 1}
    # endcap MDs store no curvature estimate
    assert np.all(r.md_kappa[ec] == 0.0)


# ------------------------------------------------------------------ brute force
@pytest.mark.parametrize("kind,index", [("toy", 0), ("toy", 1), ("pu", 0), ("pu", 1)])
def test_indexed_equals_brute_force(geom_toy, geom_full, cuts, kind, index):
    if kind == "toy":
        g, e = geom_toy, synth.toy_event(geom_toy, index)
    else:
        g = geom_full
        e = synth.pileup_event(g, index, pileup=3, mean_per_vertex=96)
    a = _run(g, e, cuts)
    b = _run(g, e, cuts, brute=True)
    for name in ("md_hits", "ls_hits", "t3_hits", "t5_hits"):
        sa = {tuple(t) for t in getattr(a, name)()}
        sb = {tuple(t) for t in getattr(b, name)()}
        assert sa == sb, name
    assert b.pairs[1] >= a.pairs[1]
    assert a.counts["t5"] > 0


# ------------------------------------------------------------------ efficiency on muons
def test_toy_muon_efficiency(geom_toy, cuts):
    found_md = total_md = 0
    denom = found = 0
    for idx in range(6):
        e = synth.toy_event(geom_toy, idx)
        r = _run(geom_toy, e, cuts)
        mdset = {tuple(t) for t in r.md_hits()}
        npart = len(e.particles["pt"])
        for p in range(npart):
            for pairs in _true_layers(geom_toy, e, p).values():
                for lo, up, _ in pairs:
                    total_md += 1
                    found_md += (lo, up) in mdset
        good = truth.findable_t5(e.sensor, e.pid, geom_toy.layer, npart)
        m = truth.match_particle(r.t5_hits(), e.pid)
        denom += good.size
        found += np.isin(good, m[m >= 0]).sum()
    assert found_md / total_md >= 0.99
    assert denom >= 200
    assert found / denom >= 0.99


def test_invalid_hits_rejected(geom_toy, cuts):
    e = synth.toy_event(geom_toy, 0)
    e.sensor[3] = geom_toy.n_sensor + 5
    with pytest.raises(ValueError):
        _run(geom_toy, e, cuts)
