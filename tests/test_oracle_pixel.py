"""Pins of the oracle's pixel-seed steps (Table 1 steps 0 and 5-8) against closed-form helices
and hand-made seed lists.

* A noiseless helix gives a seed on the four pixel cylinders and outer-tracker objects on
  the same circle: each isolated track ends as exactly one pT5, its seed matched to its own
  quintuplet, with an rz residual at the rounding level; a track too short for a T5 but with
  a T3 ends as a pT3; a seed with no outer object stays a pLS; a T5 without a seed stays a T5.
* Each matching condition is moved across its boundary on an exact helix (the azimuth and
  slope windows, the two curvature tests, the rz interpolation), with the parameter set just
  inside or just outside the value the geometry fixes.
* The one-to-one preference: of two seeds on one track the better-fitting one takes the T5.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import synth, truth

PC = synth.default_pixel_cuts()


def _run(g, e, seeds, cuts, pc=PC):
    """The oracle with every T5 selected (working point 0), so that the track-candidate T5s
    are the T5s left by the duplicate removal."""
    c = dict(cuts, wp=np.float32(0.0))
    return oracle.run_event(g, e, c, synth.mlp_flat(synth.xavier_mlp()), 2, pls=seeds, pcuts=pc)


def _noiseless_seeds(e):
    return synth.pixel_seeds(e, fake_frac=0.0, sigma_rphi=0.0, sigma_z=0.0)


def _types(r):
    t = r.pix_tc[:, 0]
    return {k: int((t == k).sum()) for k in (5, 6, 7, 8)}


@pytest.mark.parametrize("pt,eta,q", [(1.2, 0.3, 1.0), (5.0, -0.8, -1.0), (0.9, 1.6, -1.0), (20.0, 2.0, 1.0)])
def test_isolated_track_becomes_one_pt5(geom_full, cuts, pt, eta, q):
    e = synth.muon_event(geom_full, [pt], [eta], [0.4], [q], sigma=0.0)
    s = _noiseless_seeds(e)
    assert s.n == 1
    r = _run(geom_full, e, s.hits, cuts)
    ty = _types(r)
    assert ty[5] == 1 and ty[8] == 0, ty
    (typ, p, o), = [row for row in r.pix_tc.tolist() if row[0] == 5]
    assert truth.match_particle(r.t5_hits()[o:o + 1], e.pid)[0] == 0
    # the seed lies on the track's circle: the match statistics are at the rounding level
    md0, md1 = r.t5_md[o, 0], r.t5_md[o, 1]
    P = [np.array([e.x[r.md_lo[m]], e.y[r.md_lo[m]], e.z[r.md_lo[m]],
                   np.sqrt(np.float32(e.x[r.md_lo[m]]) ** 2 + np.float32(e.y[r.md_lo[m]]) ** 2)], np.float32)
         for m in (md0, md1)]
    ok, res, dk = oracle.pixel_match(s.hits[0], P[0], P[1], r.t3_kappa[r.t5_t3a[o]], PC)
    assert ok and res < 2e-3 and dk < 2e-4 * abs(float(r.t3_kappa[r.t5_t3a[o]])) + 1e-6


def test_t5_without_seed_and_seed_without_object(geom_full, cuts):
    e = synth.muon_event(geom_full, [3.0, 2.0], [0.2, -0.5], [0.3, 2.4], [1.0, -1.0], sigma=0.0)
    s = _noiseless_seeds(e)
    assert s.n == 2
    # only the first track's seed, plus a seed far from both tracks (rotated by 2 rad)
    keep = s.hits[s.pid == 0]
    c, sn = math.cos(2.0), math.sin(2.0)
    far = keep.copy()
    far[..., 0], far[..., 1] = c * keep[..., 0] - sn * keep[..., 1], sn * keep[..., 0] + c * keep[..., 1]
    r = _run(geom_full, e, np.concatenate([keep, far]), cuts)
    ty = _types(r)
    assert ty == {5: 1, 6: 1, 7: 0, 8: 1}, ty
    pls_rows = [row for row in r.pix_tc.tolist() if row[0] == 8]
    assert pls_rows[0][1] == 1 and pls_rows[0][2] == -1
    t6 = [row for row in r.pix_tc.tolist() if row[0] == 6]
    assert truth.match_particle(r.t5_hits()[t6[0][2]:t6[0][2] + 1], e.pid)[0] == 1


def test_short_track_becomes_pt3(geom_full, cuts):
    """A track with T3s but no T5: its seed ends as a pT3."""
    # a forward track through barrel layer 1 and disks 1, 2, 4, 5 (it passes between the
    # modules of disk 3): LSs and T3s but no chain of five MDs
    e = synth.muon_event(geom_full, [20.0], [2.2], [0.4], [1.0], sigma=0.0)
    r0 = oracle.run_event(geom_full, e, cuts)
    assert r0.counts["t5"] == 0 and r0.counts["t3"] > 0
    s = _noiseless_seeds(e)
    r = _run(geom_full, e, s.hits, cuts)
    ty = _types(r)
    assert ty[5] == 0 and ty[7] == 1 and ty[8] == 0, ty


def _helix_case(pt=1.0, eta=0.4, q=1.0):
    """Seed hits and the first two anchors of a noiseless barrel track with its true
    curvature (geometry of a single muon; anchors on layers 1 and 2)."""
    g = synth.build_geometry(True)
    e = synth.muon_event(g, [pt], [eta], [0.9], [q], sigma=0.0)
    s = _noiseless_seeds(e)
    lay = {}
    for m in np.unique(e.sensor // 2):
        lo = np.nonzero(e.sensor == 2 * m)[0]
        if lo.size:
            lay.setdefault(int(g.layer[m]), int(lo[0]))
    P = []
    for l in (1, 2):
        i = lay[l]
        x, y, z = np.float32(e.x[i]), np.float32(e.y[i]), np.float32(e.z[i])
        P.append(np.array([x, y, z, np.sqrt(x * x + y * y)], np.float32))
    kappa = np.float32(-q * synth.K_FIELD / pt)
    return s.hits[0], P[0], P[1], kappa


def _dphi(H4, P0):
    return math.acos((float(H4[0]) * float(P0[0]) + float(H4[1]) * float(P0[1]))
                     / (math.hypot(float(H4[0]), float(H4[1])) * float(P0[3])))


def test_azimuth_window_boundary():
    """The sine of the azimuth turn from H4 to P0 is bounded by dphi0 + dphi_cm (r0 - r4):
    each term alone is set just above or below the value this helix needs; a first anchor
    on the far side of the beamline (same sine, negative cosine) is always rejected."""
    H, P0, P1, k = _helix_case(pt=0.85, eta=0.2)
    sdphi = math.sin(_dphi(H[3], P0))
    dr = float(P0[3]) - math.hypot(float(H[3, 0]), float(H[3, 1]))
    assert sdphi > 0.02 and dr > 5.0
    for f, inside in ((1.02, True), (0.98, False)):
        pc = dict(PC, dphi0=np.float32(0.0), dphi_cm=np.float32(sdphi / dr * f))
        assert oracle.pixel_match(H, P0, P1, k, pc)[0] == inside, ("per cm", f)
        pc = dict(PC, dphi0=np.float32(sdphi * f), dphi_cm=np.float32(0.0))
        assert oracle.pixel_match(H, P0, P1, k, pc)[0] == inside, ("constant", f)
    Q = H.copy()
    Q[:, :2] = -Q[:, :2]                   # the seed mirrored through the beamline
    pc = dict(PC, dphi0=np.float32(1.0), kappa_rel=np.float32(10.0), kappa_abs=np.float32(1.0),
              rz_tol=np.float32(100.0), dm_abs=np.float32(100.0))
    assert oracle.pixel_match(H, P0, P1, k, pc)[0] and not oracle.pixel_match(Q, P0, P1, k, pc)[0]


def test_slope_window_boundary():
    H, P0, P1, k = _helix_case(pt=0.85, eta=1.0)
    r1 = math.hypot(float(H[0, 0]), float(H[0, 1]))
    r4 = math.hypot(float(H[3, 0]), float(H[3, 1]))
    mp = (float(H[3, 2]) - float(H[0, 2])) / (r4 - r1)
    mo = (float(P1[2]) - float(P0[2])) / (float(P1[3]) - float(P0[3]))
    gap = abs(mp - mo)
    assert gap > 1e-3
    for f, inside in ((1.02, True), (0.98, False)):
        pc = dict(PC, dm_abs=np.float32(gap * f), dm_rel=np.float32(0.0))
        assert oracle.pixel_match(H, P0, P1, k, pc)[0] == inside, f


def _curv3(A, B, C):
    ax, ay = B[0] - A[0], B[1] - A[1]
    bx, by = C[0] - B[0], C[1] - B[1]
    cx, cy = C[0] - A[0], C[1] - A[1]
    return 2.0 * (ax * cy - ay * cx) / (math.hypot(ax, ay) * math.hypot(bx, by) * math.hypot(cx, cy))


def _moved_to_curvature(A, M, C, target):
    """M moved perpendicular to the chord A -> C until the circle through A, M, C has the
    signed curvature `target` (float64 bisection on the offset)."""
    A, M, C = (np.asarray(v, np.float64) for v in (A, M, C))
    ux, uy = C[0] - A[0], C[1] - A[1]
    n = np.array([-uy, ux]) / math.hypot(ux, uy)
    f = lambda d: _curv3(A, (M[0] + d * n[0], M[1] + d * n[1]), C) - target
    lo, hi = -2.0, 2.0
    assert f(lo) * f(hi) < 0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(lo) * f(mid) > 0 else (lo, mid)
    d = 0.5 * (lo + hi)
    return M[0] + d * n[0], M[1] + d * n[1]


@pytest.mark.parametrize("which", ["seed", "circle"])
def test_curvature_tolerance_boundary(which):
    """One curvature is moved away from the object's ko (the true value) until it crosses
    rel (|k| + |ko|) / 2 + abs: the seed's own curvature through H1, H3, H4 (moving H3; the
    pT test) or the curvature through H1, H4, P0 (moving P0; the circle test). The other
    conditions keep holding."""
    H, P0, P1, k = _helix_case(pt=2.0, eta=0.1)
    rel, ab = float(PC["kappa_rel"]), float(PC["kappa_abs"])
    a = abs(float(k))
    hi = (a * (1 + rel / 2) + ab) / (1 - rel / 2)      # |k'| above |ko| at the boundary
    pc = dict(PC, rz_tol=np.float32(1.0))
    for f, inside in ((0.98, True), (1.02, False)):
        target = math.copysign(hi * f, float(k))
        Q, R0 = H.copy(), P0.copy()
        if which == "seed":
            x, y = _moved_to_curvature(H[0], H[2], H[3], target)
            Q[2, 0], Q[2, 1] = np.float32(x), np.float32(y)
        else:
            # the circle through H1, P0, H4 in that order has the opposite orientation
            x, y = _moved_to_curvature(H[0], P0, H[3], -target)
            R0[0], R0[1] = np.float32(x), np.float32(y)
            R0[3] = np.sqrt(R0[0] * R0[0] + R0[1] * R0[1], dtype=np.float32)
        assert oracle.pixel_match(Q, R0, P1, k, pc)[0] == inside, (which, f)


def test_rz_interpolation_boundary():
    H, P0, P1, k = _helix_case(pt=3.0, eta=0.6)
    ok, res0, _ = oracle.pixel_match(H, P0, P1, k, PC)
    assert ok and res0 < 1e-3
    tol = float(PC["rz_tol"])
    for d, inside in ((0.98 * tol, True), (1.02 * tol, False)):
        for sgn in (1.0, -1.0):
            Q = H.copy()
            Q[3, 2] = np.float32(float(H[3, 2]) + sgn * d)
            # moving z4 also moves the seed's slope; the slope window is opened for this test
            pc = dict(PC, dm_abs=np.float32(10.0))
            got, res, _ = oracle.pixel_match(Q, P0, P1, k, pc)
            assert got == inside, (d, sgn, res)


def test_better_seed_takes_the_quintuplet(geom_full, cuts):
    """Two seeds on one track, one with its outer hit moved by 0.02 cm in z: the exact one
    becomes the pT5 whatever the order of the seeds; the other does not take that T5."""
    e = synth.muon_event(geom_full, [4.0], [0.3], [1.2], [1.0], sigma=0.0)
    s = _noiseless_seeds(e)
    worse = s.hits.copy()
    worse[0, 3, 2] += np.float32(0.02)
    for seeds, best in ((np.concatenate([s.hits, worse]), 0), (np.concatenate([worse, s.hits]), 1)):
        r = _run(geom_full, e, seeds, cuts)
        pt5 = [row for row in r.pix_tc.tolist() if row[0] == 5]
        assert len(pt5) == 1 and pt5[0][1] == best
        assert all(row[1] != best for row in r.pix_tc.tolist() if row[0] in (7, 8))


def test_pixel_steps_on_pileup(geom_full, cuts):
    """On a pile-up slice: every track-candidate T5 appears once (as a pT5 or a T5), every
    seed once (in a pT5, a pT3 or as a pLS), no object twice; nearly all pT5s pair a seed
    with its own particle's T5, and fake seeds are never pT5s of a real particle's T5 with
    a wrong pairing of more than a few per mille."""
    e = synth.pileup_event(geom_full, 5, pileup=20, mean_per_vertex=96)
    s = synth.pixel_seeds(e)
    r = _run(geom_full, e, s.hits, cuts)
    rows = r.pix_tc
    t = rows[:, 0]
    t5_ids = rows[(t == 5) | (t == 6), 2]
    assert sorted(t5_ids.tolist()) == sorted(np.flatnonzero(r.t5_tc).tolist())
    seeds_used = rows[t != 6, 1]
    assert sorted(seeds_used.tolist()) == list(range(s.n))
    assert len(set(rows[t == 7, 2].tolist())) == int((t == 7).sum())
    m5 = truth.match_particle(r.t5_hits(), e.pid)
    good = [s.pid[p] == m5[o] for typ, p, o in rows.tolist() if typ == 5]
    assert len(good) > 0.9 * int(r.t5_tc.sum()) and np.mean(good) > 0.995
    # a pT3's T3 is never made entirely of MDs of pT5 quintuplets
    inpt5 = np.zeros(len(r.md_lo), bool)
    for typ, p, o in rows.tolist():
        if typ == 5:
            inpt5[r.t5_md[o]] = True
    for typ, p, o in rows.tolist():
        if typ == 7:
            assert not inpt5[r.t3_md[o]].all()
