"""Pins of the oracle's cut thresholds against closed-form geometry.

Each test builds anchors on exact circles in the transverse plane (no smearing), moves one
quantity across the boundary a cut is meant to draw, and checks that the oracle accepts
just inside it and rejects just outside (1% on either side). The expected boundary comes
from the geometry of a circle through the beamline and the error model of the cut set
(Section 1: objects "consistent with a continuous, helical trajectory", MDs with pT above
0.8 GeV; the tolerances are 3-sigma two-hit errors e over the lever arm of each estimate):

* LS curvature consistency (inner and outer MD): the direction of a barrel MD may turn
  away from the helix tangent until the sine of its angle to the radial direction has moved
  by e/g (the MD's own 3-sigma direction error over the sensor gap g) plus the segment's
  direction error e/dT scaled to the MD's radius;
* endcap MD bend: the transverse direction of an endcap MD may turn away from the radial
  direction until it exceeds the bend angle of a 0.8 GeV track from the beamline at that
  radius by a lateral 3-sigma error e over the MD's transverse step;
* T3 pT: a triplet is kept iff its circle has a radius of at least 1/(1.25 kappa_max),
  i.e. pT >= 0.64 GeV, whatever the circle's position;
* T5 curvature: two triplets are joined iff their curvatures differ by at most 30% of
  their mean plus 0.001/cm.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import synth


def _f(c, k):
    return float(np.float32(c[k]))


def _anchor(x, y, z):
    """Float32 hit (x, y, z, r) with r = sqrtf(x*x + y*y) in float32, as hits are stored."""
    x, y, z = np.float32(x), np.float32(y), np.float32(z)
    r = np.sqrt(np.float32(x * x) + np.float32(y * y), dtype=np.float32)
    return np.array([x, y, z, r], np.float32)


def _origin_circle(kappa, t, phi0=0.0):
    """Point at arc length t on the circle through the origin that leaves it in direction
    phi0 with signed curvature kappa (counter-clockwise for kappa > 0)."""
    if kappa == 0.0:
        return t * math.cos(phi0), t * math.sin(phi0)
    x, y = math.sin(kappa * t) / kappa, (1.0 - math.cos(kappa * t)) / kappa
    c, s = math.cos(phi0), math.sin(phi0)
    return c * x - s * y, s * x + c * y


def _arc_at_radius(kappa, r):
    """Arc length from the origin at which that circle reaches radius r (r = 2 sin(kt/2)/k)."""
    return 2.0 * math.asin(0.5 * r * kappa) / kappa


def _grid(star, lo=0.2, hi=1.8, n=33):
    """Scan points on both sides of a threshold, skipping the +-1% band around it."""
    f = np.linspace(lo, hi, n)
    return [(star * v, v < 0.99) for v in f if abs(v - 1.0) > 0.01]


# ------------------------------------------------------------------ LS curvature consistency
def _barrel_md(kappa, t, phi0, lam, tilt, gap):
    """Barrel MD on a helix through the origin (z = lam * arc length): lower hit at arc t,
    upper hit one sensor gap further out along the tangent turned by `tilt` radians."""
    x, y = _origin_circle(kappa, t, phi0)
    alpha = 0.5 * kappa * t                   # angle between radial direction and tangent
    theta = phi0 + kappa * t                  # tangent direction
    ell = gap / math.cos(alpha)
    L = _anchor(x, y, lam * t)
    U = _anchor(x + ell * math.cos(theta + tilt), y + ell * math.sin(theta + tilt), lam * (t + ell))
    return L, U, alpha


@pytest.mark.parametrize("ra,rb", [(23.0, 36.0), (51.0, 68.0), (88.0, 110.0)])
@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("which", ["inner", "outer"])
def test_ls_kappa_consistency_boundary(cuts, ra, rb, sign, which):
    km, e, g = _f(cuts, "kappa_max"), _f(cuts, "hit_err"), _f(cuts, "sensor_gap")
    kappa, phi0, lam = sign * km / 3.0, 0.7, 0.25
    ta, tb = _arc_at_radius(kappa, ra), _arc_at_radius(kappa, rb)
    La, Ua, alpha_a = _barrel_md(kappa, ta, phi0, lam, 0.0, g)
    Lb, Ub, alpha_b = _barrel_md(kappa, tb, phi0, lam, 0.0, g)
    dT = math.hypot(float(Lb[0]) - float(La[0]), float(Lb[1]) - float(La[1]))
    # the untilted helix passes with both MD curvatures checked
    ok_a, kA = oracle.md_cut(La, Ua, 0, cuts)
    ok_b, kB = oracle.md_cut(Lb, Ub, 0, cuts)
    assert ok_a and ok_b
    ok, kls = oracle.ls_cut(La, Lb, kA, kB, 1, 1, cuts)
    assert ok and abs(float(kls) - kappa) < 1e-4 * abs(kappa)
    # direction budget of the tilted MD, in the sine of its angle to the radial direction
    if which == "inner":
        alpha, t_md, r_md, budget = alpha_a, ta, ra, e / g + (e / dT) * (ra / rb)
    else:
        alpha, t_md, r_md, budget = alpha_b, tb, rb, e / g + e / dT
    for side in (1.0, -1.0):
        star = math.asin(math.sin(alpha) + side * budget) - alpha
        for tilt, inside in _grid(star):
            L, U, _ = _barrel_md(kappa, t_md, phi0, lam, tilt, g)
            ok_md, k_md = oracle.md_cut(L, U, 0, cuts)
            assert ok_md, (tilt, "the MD itself must pass for the scan to probe the LS cut")
            if which == "inner":
                got, _ = oracle.ls_cut(L, Lb, k_md, 0.0, 1, 0, cuts)
            else:
                got, _ = oracle.ls_cut(La, L, 0.0, k_md, 0, 1, cuts)
            assert got == inside, (which, side, tilt / star)
        # the same tilts with the curvature check switched off (an endcap MD) all pass
        L, U, _ = _barrel_md(kappa, t_md, phi0, lam, 1.8 * star, g)
        k_md = oracle.md_cut(L, U, 0, cuts)[1]
        args = (L, Lb, k_md, 0.0, 0, 0) if which == "inner" else (La, L, 0.0, k_md, 0, 0)
        assert oracle.ls_cut(*args, cuts)[0]


def test_ls_kappa_pt_threshold_helices(geom_toy, cuts):
    """Noiseless helices just above 0.8 GeV keep every layer-to-layer segment with both
    barrel MD curvatures checked, each MD's curvature taken from its own two hits."""
    for q in (-1.0, 1.0):
        e = synth.muon_event(geom_toy, [0.8 * 1.05], [0.1], [1.1], [q], sigma=0.0)
        mods = {}
        for m in np.unique(e.sensor // 2):
            lo = np.nonzero(e.sensor == 2 * m)[0]
            up = np.nonzero(e.sensor == 2 * m + 1)[0]
            if lo.size and up.size:
                mods.setdefault(int(geom_toy.layer[m]), (int(lo[0]), int(up[0])))
        pairs = [l for l in range(1, 6) if l in mods and l + 1 in mods]
        assert len(pairs) >= 4
        for l in pairs:
            md = []
            for lay in (l, l + 1):
                lo, up = mods[lay]
                L = _anchor(e.x[lo], e.y[lo], e.z[lo])
                U = _anchor(e.x[up], e.y[up], e.z[up])
                ok, k = oracle.md_cut(L, U, 0, cuts)
                assert ok
                md.append((L, k))
            ok, _ = oracle.ls_cut(md[0][0], md[1][0], md[0][1], md[1][1], 1, 1, cuts)
            assert ok, (q, l)


# ------------------------------------------------------------------ endcap MD bend
def _endcap_md(r, z, phi, alpha, gap):
    """Endcap MD whose lower hit sits at radius r on the disk at z and whose transverse step
    points alpha radians off the radial direction, sized so that its radial component is
    exactly g r / |z| (the step of a straight line from the origin)."""
    x, y = r * math.cos(phi), r * math.sin(phi)
    dT = gap * (r / abs(z)) / math.cos(alpha)
    U = (x + dT * math.cos(phi + alpha), y + dT * math.sin(phi + alpha), z + math.copysign(gap, z))
    return _anchor(x, y, z), _anchor(*U)


@pytest.mark.parametrize("r", [30.0, 60.0, 100.0])
@pytest.mark.parametrize("z", [130.0, -225.0])
def test_endcap_md_bend_boundary(cuts, r, z):
    km, e, g = _f(cuts, "kappa_max"), _f(cuts, "hit_err"), _f(cuts, "sensor_gap")
    alpha_max = math.asin(0.5 * r * km)        # bend angle of a 0.8 GeV track at radius r
    star = math.atan(math.tan(alpha_max) + e * abs(z) / (g * r))
    for phi in (0.3, 2.5, -1.7):
        for sgn in (1.0, -1.0):
            for a, inside in _grid(star, hi=min(1.8, 1.45 / star)):
                L, U = _endcap_md(r, z, phi, sgn * a, g)
                ok, k = oracle.md_cut(L, U, 1, cuts)
                assert ok == inside, (r, z, phi, sgn, a / star)
                if ok:
                    assert k == 0.0


def _helix_endcap_md(pt, q, r, zd, gap):
    """Lower and upper hit of a noiseless helix from the origin (pT, charge q) crossing the
    two sensor planes of a disk at |z| = zd, tuned to reach radius r at the disk."""
    kappa = -q * synth.K_FIELD / pt
    t = _arc_at_radius(kappa, r)
    lam = zd / t
    out = []
    for zz in (zd - 0.5 * gap, zd + 0.5 * gap):
        x, y = _origin_circle(kappa, zz / lam, 0.4)
        out.append(_anchor(x, y, zz))
    return out, kappa


def test_endcap_md_pt_threshold_helices(cuts):
    """Exact helices from the origin: every endcap MD of a 0.84 GeV track passes; a 0.64 GeV
    track's MDs fail wherever its bend exceeds the 0.8 GeV bend by more than twice the
    lateral error budget."""
    km, e, g = _f(cuts, "kappa_max"), _f(cuts, "hit_err"), _f(cuts, "sensor_gap")
    rejected = 0
    for zd in (130.0, 160.0, 190.0, 225.0, 265.0):
        for r in (28.0, 40.0, 55.0, 70.0, 85.0, 100.0):
            for q in (-1.0, 1.0):
                (L, U), _ = _helix_endcap_md(0.8 * 1.05, q, r, zd, g)
                assert oracle.md_cut(L, U, 1, cuts)[0], (zd, r, q)
                (L, U), kappa = _helix_endcap_md(0.8 * 0.8, q, r, zd, g)
                alpha, alpha_max = math.asin(0.5 * r * abs(kappa)), math.asin(0.5 * r * km)
                excess = g * (r / zd) * (math.tan(alpha) - math.tan(alpha_max))
                if excess > 2.0 * e:
                    assert not oracle.md_cut(L, U, 1, cuts)[0], (zd, r, q)
                    rejected += 1
    assert rejected >= 12


# ------------------------------------------------------------------ T3 pT
@pytest.mark.parametrize("sign", [1.0, -1.0])
@pytest.mark.parametrize("through_origin", [True, False])
def test_t3_pt_boundary(cuts, sign, through_origin):
    km, fac = _f(cuts, "kappa_max"), _f(cuts, "t3_kappa_factor")
    R_star = 1.0 / (fac * km)                  # pT = 0.8 / 1.25 GeV
    for f, inside in ((1.01, True), (1.05, True), (1.5, True), (0.99, False), (0.95, False), (0.7, False)):
        R = f * R_star
        kappa = sign / R
        for phi0 in (0.2, 1.9, -2.8):
            if through_origin:
                ts = [_arc_at_radius(kappa, r) for r in (23.0, 36.0, 0.95 * min(51.0, 2.0 * R))]
                pts = [_origin_circle(kappa, t, phi0) for t in ts]
            else:
                # a displaced circle: centre 35 cm from the origin, anchors 12 cm apart
                cx, cy = 35.0 * math.cos(phi0), 35.0 * math.sin(phi0)
                ang = [phi0 + sign * s / R for s in (0.0, 12.0, 24.0)]
                pts = [(cx + R * math.cos(a), cy + R * math.sin(a)) for a in ang]
            P = [_anchor(x, y, 0.1 * i) for i, (x, y) in enumerate(pts)]
            ok, k = oracle.t3_cut(P[0], P[1], P[2], cuts)
            assert ok == inside, (f, phi0)
            if ok:
                assert abs(abs(float(k)) - 1.0 / R) <= 1e-4 / R


# ------------------------------------------------------------------ T5 curvature consistency
def _two_arc_anchors(ka, kb, phi0):
    """Five anchors: P0..P2 on a circle of curvature ka through the origin (radii 23, 36,
    51 cm), then P3, P4 continuing from P2 with the same tangent on a circle of curvature kb,
    17 and 37 cm of arc further; z = 0."""
    pts = [_origin_circle(ka, _arc_at_radius(ka, r), phi0) for r in (23.0, 36.0, 51.0)]
    t2 = _arc_at_radius(ka, 51.0)
    theta = phi0 + ka * t2
    x2, y2 = pts[2]
    for s in (17.0, 37.0):
        pts.append((x2 + (math.sin(theta + kb * s) - math.sin(theta)) / kb,
                    y2 - (math.cos(theta + kb * s) - math.cos(theta)) / kb))
    return [_anchor(x, y, 0.0) for x, y in pts]


@pytest.mark.parametrize("ka", [0.004, 0.01, -0.006])
def test_t5_kappa_consistency_boundary(cuts, ka):
    rel, ab = _f(cuts, "t5_kappa_rel"), _f(cuts, "t5_kappa_abs")
    h = 0.5 * rel
    a = abs(ka)
    hi = (a * (1.0 + h) + ab) / (1.0 - h)      # |kb| - |ka| = h (|ka| + |kb|) + ab
    lo = (a * (1.0 - h) - ab) / (1.0 + h)      # |ka| - |kb| = h (|ka| + |kb|) + ab
    cases = [(hi * f, f < 0.99) for f in (0.9, 0.97, 0.985, 1.015, 1.03, 1.1)]
    cases += [(lo * f, f > 1.01) for f in (0.9, 0.97, 0.985, 1.015, 1.03, 1.1)]
    for kb_abs, inside in cases:
        kb = math.copysign(kb_abs, ka)
        for phi0 in (0.3, -2.2):
            P = _two_arc_anchors(ka, kb, phi0)
            ok_a, k_a = oracle.t3_cut(P[0], P[1], P[2], cuts)
            ok_b, k_b = oracle.t3_cut(P[2], P[3], P[4], cuts)
            assert ok_a and ok_b
            assert abs(float(k_a) - ka) < 1e-4 * abs(ka) and abs(float(k_b) - kb) < 1e-3 * abs(kb)
            assert oracle.t5_cut(np.stack(P), k_a, k_b, cuts) == inside, (ka, kb / ka)


# ------------------------------------------------------------------ barrel MD bend and road
def _barrel_pair(r, zL, phi, alpha, ell, dz):
    """Barrel hit pair: lower hit at radius r, azimuth phi; upper hit ell further along a
    transverse direction alpha radians off the radial one, dz higher."""
    x, y = r * math.cos(phi), r * math.sin(phi)
    return (_anchor(x, y, zL),
            _anchor(x + ell * math.cos(phi + alpha), y + ell * math.sin(phi + alpha), zL + dz))


@pytest.mark.parametrize("r", [23.0, 51.0, 110.0])
def test_barrel_md_bend_boundary(cuts, r):
    """The MD direction may leave the radial direction until the sine of the angle exceeds
    that of a 0.8 GeV track from the beamline at this radius (r kappa_max / 2) by the 3-sigma
    direction error across the sensor gap (e / g)."""
    km, e, g = _f(cuts, "kappa_max"), _f(cuts, "hit_err"), _f(cuts, "sensor_gap")
    star = math.asin(0.5 * r * km + e / g)
    for phi in (0.4, -2.9):
        for sgn in (1.0, -1.0):
            for a, inside in _grid(star):
                L, U = _barrel_pair(r, 0.0, phi, sgn * a, g / math.cos(a), 0.0)
                ok, k = oracle.md_cut(L, U, 0, cuts)
                assert ok == inside, (r, phi, sgn, a / star)
                if ok:   # the stored curvature is 2 sin(alpha) / r with the turning sign
                    assert abs(float(k) - 2.0 * math.sin(sgn * a) / r) < 1e-4 * abs(float(k)) + 1e-7


@pytest.mark.parametrize("r", [23.0, 68.0, 110.0])
@pytest.mark.parametrize("zL", [0.0, 40.0, -90.0])
def test_barrel_md_road_boundary(cuts, r, zL):
    """The MD's r-z direction must point back to the beamline within the luminous-region
    half-length Zl of the origin; the hit error e on dz widens that to Zl + e r / dr."""
    Zl, e, g = _f(cuts, "z_lum"), _f(cuts, "hit_err"), _f(cuts, "sensor_gap")
    star = Zl + e * r / g
    for sgn in (1.0, -1.0):
        for z0, inside in _grid(star, lo=0.0, hi=1.6):
            z0 = sgn * z0
            dz = (zL - z0) / r * g          # the line through (0, z0) and the lower hit
            L, U = _barrel_pair(r, zL, 1.0, 0.0, g, dz)
            assert oracle.md_cut(L, U, 0, cuts)[0] == inside, (r, zL, z0 / star)


@pytest.mark.parametrize("r", [30.0, 80.0])
@pytest.mark.parametrize("z", [130.0, -265.0])
def test_endcap_md_road_boundary(cuts, r, z):
    """Endcap MD: the radial component of the transverse step between the two sensors must
    match that of a straight line from the origin (g r / |z|) within the change caused by
    moving the line's origin Zl along the beamline, plus e. The step is varied through the
    beamline intercept z0 of a line through the lower hit (positive towards the disk)."""
    Zl, e, g = _f(cuts, "z_lum"), _f(cuts, "hit_err"), _f(cuts, "sensor_gap")
    az = abs(z)
    step = lambda z0: g * r / (az - z0)            # radial step of the line from (0, z0)
    tol = step(Zl) - step(0.0) + e
    # intercepts at which the step differs from the origin line's by exactly tol
    hi = az - g * r / (step(0.0) + tol)
    lo = az - g * r / (step(0.0) - tol)
    for star in (hi, lo):
        for z0, inside in _grid(star, lo=0.0, hi=1.5):
            x, y = r * math.cos(0.8), r * math.sin(0.8)
            d = step(z0)
            L = _anchor(x, y, z)
            U = _anchor(x + d * math.cos(0.8), y + d * math.sin(0.8), z + math.copysign(g, z))
            assert oracle.md_cut(L, U, 1, cuts)[0] == inside, (r, z, z0, star)


def test_md_direction(cuts):
    """A track from the luminous region crosses the lower sensor first: an upper hit on the
    beamline side of the lower one is no MD (barrel), nor is an endcap pair whose z step
    points back to the interaction region."""
    g = _f(cuts, "sensor_gap")
    L, U = _barrel_pair(40.0, 10.0, 0.5, 0.0, g, 0.065)
    assert oracle.md_cut(L, U, 0, cuts)[0]
    L, U = _barrel_pair(40.0, 10.0, 0.5, math.pi, g, 0.065)
    assert not oracle.md_cut(L, U, 0, cuts)[0]
    x, y = 50.0 * math.cos(1.0), 50.0 * math.sin(1.0)
    d = g * 50.0 / 160.0
    L = _anchor(x, y, 160.0)
    U = _anchor(x + d * math.cos(1.0), y + d * math.sin(1.0), 160.0 + g)
    assert oracle.md_cut(L, U, 1, cuts)[0]
    Ub = _anchor(x + d * math.cos(1.0), y + d * math.sin(1.0), 160.0 - g)
    assert not oracle.md_cut(L, Ub, 1, cuts)[0]


# ------------------------------------------------------------------ LS bend with a short chord
@pytest.mark.parametrize("dT", [1.0, 4.0, 14.0])
@pytest.mark.parametrize("ra", [30.0, 80.0])
def test_ls_bend_boundary(cuts, dT, ra):
    """A segment's chord may leave the radial direction at its inner anchor until the sine of
    the angle exceeds the inscribed angle of a 0.8 GeV circle through the origin at the outer
    radius (rb kappa_max / 2) by the lateral 3-sigma error over the chord (e / dT). Anchors on
    a line through the origin in r-z (z0 = 0), so the luminous-region test is neutral."""
    km, e = _f(cuts, "kappa_max"), _f(cuts, "hit_err")
    phi, slope = -0.6, 1.7                  # z / r of both anchors

    def outer(beta):
        xa, ya = ra * math.cos(phi), ra * math.sin(phi)
        xb, yb = xa + dT * math.cos(phi + beta), ya + dT * math.sin(phi + beta)
        return (xa, ya), (xb, yb), math.hypot(xb, yb)

    def excess(beta):
        return math.sin(beta) - (0.5 * outer(beta)[2] * km + e / dT)

    lo_b, hi_b = 0.0, 1.5
    for _ in range(100):
        mid = 0.5 * (lo_b + hi_b)
        lo_b, hi_b = (mid, hi_b) if excess(mid) < 0 else (lo_b, mid)
    star = lo_b
    for sgn in (1.0, -1.0):
        for b, inside in _grid(star, hi=min(1.8, 1.4 / star)):
            (xa, ya), (xb, yb), rb = outer(sgn * b)
            A, B = _anchor(xa, ya, slope * ra), _anchor(xb, yb, slope * rb)
            ok, k = oracle.ls_cut(A, B, 0.0, 0.0, 0, 0, cuts)
            assert ok == inside, (dT, ra, sgn, b / star)
            if ok:   # the curvature of the circle through the origin and both anchors
                assert abs(float(k) - 2.0 * math.sin(sgn * b) / rb) < 1e-4 * abs(float(k)) + 1e-7


@pytest.mark.parametrize("ra,rb", [(23.0, 36.0), (68.0, 88.0), (100.0, 101.0), (60.0, 60.5)])
def test_ls_luminous_road_boundary(cuts, ra, rb):
    """The straight r-z line through both anchors must meet the beamline within Zl of the
    origin, widened by the anchors' error e: an error e in the inner z moves the intercept
    by e, and an error e in the z difference of the anchors moves it by e ra / (rb - ra),
    which dominates for the short radial lever arms of forward segments between disks (last
    two cases)."""
    Zl, e = _f(cuts, "z_lum"), _f(cuts, "hit_err")
    star = Zl + e + e * ra / (rb - ra)
    for sgn in (1.0, -1.0):
        for z0, inside in _grid(star, lo=0.0, hi=1.5):
            z0 = sgn * z0
            za, zb = z0 + 0.8 * ra, z0 + 0.8 * rb     # the line z = z0 + 0.8 r
            A = _anchor(ra * math.cos(0.3), ra * math.sin(0.3), za)
            B = _anchor(rb * math.cos(0.3), rb * math.sin(0.3), zb)
            assert oracle.ls_cut(A, B, 0.0, 0.0, 0, 0, cuts)[0] == inside, (ra, z0 / star)
    # a segment pointing inwards is no segment
    A = _anchor(ra * math.cos(0.3), ra * math.sin(0.3), 0.8 * ra)
    B = _anchor(rb * math.cos(0.3), rb * math.sin(0.3), 0.8 * rb)
    assert oracle.ls_cut(A, B, 0.0, 0.0, 0, 0, cuts)[0] and not oracle.ls_cut(B, A, 0.0, 0.0, 0, 0, cuts)[0]


# ------------------------------------------------------------------ r-z consistency of T3 and T5
def _helix_anchors(kappa, radii, lam, phi0):
    """Anchors of a helix through the origin at the given radii, z = lam * arc length."""
    out = []
    for r in radii:
        t = _arc_at_radius(kappa, r)
        x, y = _origin_circle(kappa, t, phi0)
        out.append(_anchor(x, y, lam * t))
    return out


@pytest.mark.parametrize("kappa,lam", [(0.009, 1.0), (-0.012, 0.6), (0.0005, 2.5), (-0.004, 3.0)])
def test_t3_rz_boundary(cuts, kappa, lam):
    """On a helix z grows linearly with arc length; the middle anchor may leave the helix in
    z by up to the tolerance. Unequal anchor spacings and strong curvature make the chord
    differ from the arc, so the arc-length correction matters at this precision: on the
    first two helices it moves the predicted z by 12-36% of the tolerance, while the terms
    beyond it (relative 3 (c kappa)^4 / 640 of an arc over a chord c) stay below 0.2%."""
    tol = _f(cuts, "t3_rz_tol")
    for radii in ((23.0, 30.0, 51.0), (51.0, 66.0, 70.0)):
        P = _helix_anchors(kappa, radii, lam, 0.9)
        assert oracle.t3_cut(P[0], P[1], P[2], cuts)[0]
        for sgn in (1.0, -1.0):
            for d, inside in _grid(tol, lo=0.5, hi=1.5, n=21):
                Q = [p.copy() for p in P]
                Q[1][2] = np.float32(float(P[1][2]) + sgn * d)
                assert oracle.t3_cut(Q[0], Q[1], Q[2], cuts)[0] == inside, (radii, sgn, d / tol)


@pytest.mark.parametrize("kappa,lam", [(0.008, 1.0), (-0.004, 2.0), (0.008, 0.4)])
def test_t5_rz_boundary(cuts, kappa, lam):
    """The three inner anchors of a T5 may each leave the helix in z by up to the tolerance
    (z linear in the arc length estimated with the mean curvature of the two T3s). The
    arc-length correction moves the prediction by 10-26% of the tolerance on these helices;
    the terms beyond it by at most 0.12%."""
    tol = _f(cuts, "t5_rz_tol")
    P = _helix_anchors(kappa, (23.0, 36.0, 51.0, 68.0, 88.0), lam, -1.3)
    ok_a, ka = oracle.t3_cut(P[0], P[1], P[2], cuts)
    ok_b, kb = oracle.t3_cut(P[2], P[3], P[4], cuts)
    assert ok_a and ok_b and oracle.t5_cut(np.stack(P), ka, kb, cuts)
    for j in (1, 2, 3):
        for sgn in (1.0, -1.0):
            for d, inside in _grid(tol, lo=0.5, hi=1.5, n=21):
                Q = [p.copy() for p in P]
                Q[j][2] = np.float32(float(P[j][2]) + sgn * d)
                assert oracle.t5_cut(np.stack(Q), ka, kb, cuts) == inside, (j, sgn, d / tol)


def test_t5_opposite_bending_never_joined(cuts):
    """A helix keeps its sense of rotation: two nearly straight triplets bending in opposite
    directions are not joined even though their curvatures differ by less than the
    curvature tolerance; the same pair with one sense is joined."""
    k = 0.0003
    P = _two_arc_anchors(k, k, 0.5)
    ka, kb = oracle.t3_cut(P[0], P[1], P[2], cuts)[1], oracle.t3_cut(P[2], P[3], P[4], cuts)[1]
    assert oracle.t5_cut(np.stack(P), ka, kb, cuts)
    P = _two_arc_anchors(k, -k, 0.5)
    ka, kb = oracle.t3_cut(P[0], P[1], P[2], cuts)[1], oracle.t3_cut(P[2], P[3], P[4], cuts)[1]
    assert float(ka) > 0.0 > float(kb)
    assert abs(float(ka) - float(kb)) < _f(cuts, "t5_kappa_abs")
    assert not oracle.t5_cut(np.stack(P), ka, kb, cuts)
