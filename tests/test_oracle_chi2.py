"""Pins of the oracle's circle-fit chi2 (the selection of the pre-DNN mode, Section 2),
each against something other than the oracle itself: exact circles, the linearised
least-squares value of a single displaced anchor (leverage from an FP64 hat matrix),
symmetries, the chi-square law with 5 - 3 = 2 degrees of freedom on single-particle
quintuplets of smeared events, and the cut semantics of the pre-DNN mode."""
import math

import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import synth, truth

SIGMA = 0.003


def arc(R, phi0, span, offset=60.0, delta=None):
    """Five points on a circle of radius R whose middle point sits ~offset cm from the
    origin (inside the tracker), optionally displaced radially by delta[i]."""
    mid = phi0 + span / 2
    cx = (offset - R) * math.cos(mid)
    cy = (offset - R) * math.sin(mid)
    ph = phi0 + np.linspace(0.0, span, 5)
    rr = R + (np.zeros(5) if delta is None else np.asarray(delta))
    P = np.zeros((5, 4))
    P[:, 0] = cx + rr * np.cos(ph)
    P[:, 1] = cy + rr * np.sin(ph)
    P[:, 3] = np.hypot(P[:, 0], P[:, 1])
    return P.astype(np.float32), ph


@pytest.mark.parametrize("R", [40.0, 70.0, 300.0, 3e3, 3e4, 1e6, 1e9])
def test_exact_circles_of_any_radius(R):
    span = min(80.0 / R, 1.5)
    worst = max(float(oracle.t5_chi2(arc(R, phi0, span)[0], SIGMA))
                for phi0 in np.linspace(0.0, 2 * math.pi, 17))
    assert worst < 1e-3, worst          # FP32 rounding of 100 cm coordinates is ~0.002 sigma


@pytest.mark.parametrize("R", [60.0, 300.0])
@pytest.mark.parametrize("j", range(5))
@pytest.mark.parametrize("phi0", [0.3, 1.9, 4.0])
def test_single_displaced_anchor_gives_the_linearised_value(R, j, phi0):
    """chi2 of a least-squares circle after moving point j by k sigma radially is
    k^2 (1 - h_jj), h = J (J^T J)^-1 J^T, J = d(distance)/d(centre, radius)."""
    span = min(80.0 / R, 1.5)
    k = 3.0
    delta = np.zeros(5)
    delta[j] = k * SIGMA
    P, ph = arc(R, phi0, span, delta=delta)
    J = np.stack([-np.cos(ph), -np.sin(ph), -np.ones(5)], 1)
    h = J @ np.linalg.inv(J.T @ J) @ J.T
    expect = k * k * (1.0 - h[j, j])
    got = float(oracle.t5_chi2(P, SIGMA))
    assert abs(got - expect) <= 0.01 * expect + 2e-3, (got, expect)


def test_symmetries_and_sigma_scaling():
    rng = np.random.default_rng(3)
    P, _ = arc(150.0, 0.7, 80.0 / 150.0)
    P[:, :2] += rng.normal(0.0, SIGMA, (5, 2)).astype(np.float32)
    c = float(oracle.t5_chi2(P, SIGMA))
    assert c > 0.05
    rot = P.copy()
    rot[:, 0], rot[:, 1] = -P[:, 1], P[:, 0]          # exact 90 degree rotation
    mir = P.copy()
    mir[:, 1] = -P[:, 1]                              # mirror (opposite charge)
    rev = P[::-1].copy()                              # traversed backwards
    for Q in (rot, mir, rev):
        assert abs(float(oracle.t5_chi2(Q, SIGMA)) - c) <= 1e-3 * c + 1e-4
    assert abs(float(oracle.t5_chi2(P, SIGMA / 2)) - 4 * c) <= 1e-5 * c


def test_degenerate_anchors_fail_any_cut():
    P, _ = arc(100.0, 0.2, 0.8)
    P[1] = P[0]
    P[3] = P[0]
    P[4] = P[0]                                       # only two distinct points
    c = float(oracle.t5_chi2(P, SIGMA))
    assert not (c <= 1e30)                            # inf or NaN: no chi2 cut passes


@pytest.fixture(scope="module")
def pu200_open():
    g = synth.build_geometry(True)
    e = synth.pileup_event(g, 100, pileup=200, mean_per_vertex=96, config=3)
    ref = oracle.run_event(g, e, synth.open_cuts(), None)
    return g, e, ref


def test_chi_square_law_with_two_degrees_of_freedom(pu200_open):
    """Anchors of single-particle quintuplets carry independent Gaussian errors of sigma
    across the track (30 um in the sensor plane, no material), so chi2 follows the
    chi-square law with 2 degrees of freedom: CDF 1 - exp(-x/2)."""
    _, e, ref = pu200_open
    hits = ref.t5_hits()
    m = truth.match_particle(hits, e.pid)
    pure = (m >= 0) & (e.pid[hits] == m[:, None]).all(1)
    c = np.sort(ref.t5_chi2[pure].astype(np.float64))
    assert len(c) > 20_000
    cdf = 1.0 - np.exp(-c / 2.0)
    emp = np.arange(1, len(c) + 1) / len(c)
    ks = float(np.max(np.abs(emp - cdf)))
    assert ks < 0.03, ks
    assert abs(np.median(c) - 2.0 * math.log(2.0)) < 0.1


def test_pre_dnn_mode_keeps_exactly_the_quintuplets_under_the_chi2_bound(pu200_open):
    g, e, ref_open = pu200_open
    for chi2_max in (5.0, 20.0):
        ref = oracle.run_event(g, e, synth.pre_dnn_cuts(chi2_max), None)
        keep = ref_open.t5_chi2 <= np.float32(chi2_max)
        a = ref.t5_hits()
        b = ref_open.t5_hits()[keep]
        assert len(a) == len(b) and 0 < len(a) < len(ref_open.t5_chi2)
        assert np.array_equal(a[np.lexsort(a.T[::-1])], b[np.lexsort(b.T[::-1])])
        assert np.array_equal(ref.t5_chi2[np.lexsort(a.T[::-1])], ref_open.t5_chi2[keep][np.lexsort(b.T[::-1])])
