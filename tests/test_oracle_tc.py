"""Pins of the oracle's track-candidate step: selected T5s cleaned of duplicates (two T5s
sharing >= 3 of their 5 MDs; the one with the smaller circle-fit chi2, then the smaller
hit tuple, ranks above; one pass). Hand-built T5 sets fix the semantics; index == brute
force; the kept set holds no duplicates; isolated muons give one candidate each."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import synth, truth


def build(mds, q, sel=None, keys=None):
    md = np.asarray(mds, np.int32)
    n = len(md)
    if keys is None:
        keys = np.stack([np.repeat(md, 2, axis=1)[i] * 2 + np.tile([0, 1], 5) for i in range(n)])
    sel = np.ones(n, np.uint8) if sel is None else np.asarray(sel, np.uint8)
    q = np.asarray(q, np.float32)
    a = oracle.tc_select(md, keys, q, sel, int(md.max()) + 1)
    b = oracle.tc_select(md, keys, q, sel, int(md.max()) + 1, brute=True)
    assert np.array_equal(a, b)
    return list(a)


def test_three_shared_mds_make_a_duplicate():
    assert build([[0, 1, 2, 3, 4], [2, 3, 4, 5, 6]], [1.0, 2.0]) == [1, 0]
    assert build([[0, 1, 2, 3, 4], [2, 3, 4, 5, 6]], [2.0, 1.0]) == [0, 1]


def test_two_shared_mds_are_not_a_duplicate():
    assert build([[0, 1, 2, 3, 4], [3, 4, 5, 6, 7]], [1.0, 2.0]) == [1, 1]


def test_one_pass_semantics_on_a_chain():
    # A ~ B (MDs 2,3,4), B ~ C (MDs 4,5,6), A and C share one MD: B is removed by A and C by
    # B, although B itself is not a track candidate
    assert build([[0, 1, 2, 3, 4], [2, 3, 4, 5, 6], [4, 5, 6, 7, 8]], [1.0, 2.0, 3.0]) == [1, 0, 0]


def test_ties_go_to_the_smaller_hit_tuple():
    md = [[0, 1, 2, 3, 4], [0, 1, 2, 3, 5]]
    k = np.array([[10] * 10, [10] * 9 + [9]], np.int32)
    assert build(md, [1.0, 1.0], keys=k) == [0, 1]
    k2 = np.array([[10] * 9 + [9], [10] * 10], np.int32)
    assert build(md, [1.0, 1.0], keys=k2) == [1, 0]


def test_nan_counts_as_infinity():
    md = [[0, 1, 2, 3, 4], [0, 1, 2, 3, 5]]
    assert build(md, [np.nan, 5.0]) == [0, 1]
    assert build(md, [5.0, np.nan]) == [1, 0]
    # NaN and +inf tie: the hit tuple decides
    k = np.array([[10] * 10, [10] * 9 + [9]], np.int32)
    assert build(md, [np.nan, np.inf], keys=k) == [0, 1]


def test_unselected_t5s_neither_survive_nor_remove():
    md = [[0, 1, 2, 3, 4], [2, 3, 4, 5, 6]]
    assert build(md, [1.0, 2.0], sel=[0, 1]) == [0, 1]


def test_index_equals_brute_force_on_random_sets():
    rng = np.random.default_rng(7)
    for _ in range(20):
        n = int(rng.integers(1, 300))
        md = np.array([rng.choice(40, 5, replace=False) for _ in range(n)], np.int32)
        keys = rng.integers(0, 50, (n, 10)).astype(np.int32)
        q = rng.choice([0.5, 1.0, 2.0, np.nan, np.inf], n).astype(np.float32)
        sel = (rng.uniform(size=n) < 0.8).astype(np.uint8)
        a = oracle.tc_select(md, keys, q, sel, 40)
        b = oracle.tc_select(md, keys, q, sel, 40, brute=True)
        assert np.array_equal(a, b)


def test_event_index_equals_brute_force(geom_toy, cuts):
    every = dict(cuts, wp=np.float32(0.0))        # no network: every T5 is selected
    e = synth.toy_event(geom_toy, 4)
    a = oracle.run_event(geom_toy, e, every, None)
    b = oracle.run_event(geom_toy, e, every, None, brute=True)
    assert 0 < len(a.tc_hits()) < len(a.t5_md)
    assert np.array_equal(np.sort(a.tc_hits(), axis=0), np.sort(b.tc_hits(), axis=0))


@pytest.fixture(scope="module")
def pu_open():
    g = synth.build_geometry(True)
    e = synth.pileup_event(g, 102, pileup=100, mean_per_vertex=96, config=3)
    return e, oracle.run_event(g, e, synth.pre_dnn_cuts(20.0), None)


def test_kept_set_has_no_duplicates_and_every_removal_has_a_reason(pu_open):
    _, r = pu_open
    md, tc, sel = r.t5_md, r.t5_tc.astype(bool), r.t5_sel.astype(bool)
    assert sel.all() and 0 < tc.sum() < len(tc)
    by_md = {}
    for t in np.flatnonzero(sel):
        for m in md[t]:
            by_md.setdefault(int(m), []).append(int(t))
    key = r.t5_hits()
    q = np.where(np.isnan(r.t5_chi2), np.inf, r.t5_chi2)

    def above(u, t):
        return q[u] < q[t] or (q[u] == q[t] and tuple(key[u]) < tuple(key[t]))

    for t in np.flatnonzero(sel):
        dups = {u for m in md[t] for u in by_md[int(m)] if u != t and len(set(md[u]) & set(md[t])) >= 3}
        if tc[t]:
            assert not any(tc[u] for u in dups)          # no two kept T5s are duplicates
            assert not any(above(u, t) for u in dups)
        else:
            assert any(above(u, t) for u in dups)        # removed only by a better duplicate


def test_one_track_candidate_per_isolated_muon(geom_toy, cuts):
    every = dict(cuts, wp=np.float32(0.0))        # no network: every T5 is selected
    n_one = n_found = n_tc = n_fake = 0
    for index in range(5):
        e = synth.toy_event(geom_toy, index)
        r = oracle.run_event(geom_toy, e, every, None)
        m = truth.match_particle(r.tc_hits(), e.pid)
        n_tc += len(m)
        n_fake += int(np.sum(m < 0))
        found = truth.findable_t5(e.sensor, e.pid, geom_toy.layer, int(e.pid.max()) + 1)
        for p in found:
            k = int(np.sum(m == p))
            n_found += 1
            n_one += k == 1
    assert n_found > 150
    assert n_one >= 0.95 * n_found, (n_one, n_found)
    assert n_fake <= 0.02 * n_tc
