"""Pins of the oracle's T5-DNN features and forward pass (Section 2).

Features are checked against analytic helix quantities of noiseless tracks (so a
permuted, rescaled or mis-signed feature fails); the network against hand-solvable
weight sets (so a transposed weight matrix, a missing bias or a missing ReLU fails)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import synth, truth

NF, NH = 38, 32
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _zero_mlp(n_hidden=2):
    return {"W": [np.zeros((NH, NF))] + [np.zeros((NH, NH))] * (n_hidden - 1) + [np.zeros((1, NH))],
            "b": [np.zeros(NH)] * n_hidden + [np.zeros(1)]}


def test_paper_facts_fixture():
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    assert facts["n_inputs"]["value"] == NF
    assert facts["hidden_width"]["value"] == NH
    assert facts["hidden_layers"]["value"] == 2
    assert synth.mlp_hidden_layers(synth.xavier_mlp()) == 2
    # the MD pT threshold sets the curvature bound of the cut parameters
    c = synth.default_cuts()
    assert abs(float(c["kappa_max"]) - synth.K_FIELD / facts["md_pt_min_gev"]["value"]) < 1e-8


@pytest.mark.parametrize("n_hidden", [1, 2, 3, 4])
def test_zero_network_gives_one_half(n_hidden):
    f = np.linspace(-1, 1, NF)
    assert oracle.mlp_forward(synth.mlp_flat(_zero_mlp(n_hidden)), n_hidden, f) == 0.5


def test_output_bias_only():
    m = _zero_mlp()
    m["b"][-1] = np.array([math.log(3.0)])
    assert abs(oracle.mlp_forward(synth.mlp_flat(m), 2, np.ones(NF)) - 0.75) < 1e-15


@pytest.mark.parametrize("n_hidden", [1, 2, 3, 4])
def test_single_path_network(n_hidden):
    # one path feature 7 -> hidden unit 3 -> ... -> hidden unit 11 -> output; W[out, in]
    m = _zero_mlp(n_hidden)
    m["W"][0] = np.zeros((NH, NF)); m["W"][0][3, 7] = 0.5
    m["b"][0] = np.zeros(NH); m["b"][0][3] = 0.25
    prev = 3
    for l in range(1, n_hidden):
        W = np.zeros((NH, NH)); W[11, prev] = 2.0
        m["W"][l] = W
        prev = 11
    wo = np.zeros((1, NH)); wo[0, prev] = -1.5
    m["W"][-1] = wo
    f = np.zeros(NF); f[7] = 3.0; f[3] = -10.0; f[11] = 5.0
    h = max(0.0, 0.5 * 3.0 + 0.25) * (2.0 ** (n_hidden - 1))
    expect = 1.0 / (1.0 + math.exp(1.5 * h))
    got = oracle.mlp_forward(synth.mlp_flat(m), n_hidden, f)
    assert abs(got - expect) < 1e-15
    # the ReLU cuts a negative pre-activation: the output drops to sigmoid(0)
    f[7] = -3.0
    assert oracle.mlp_forward(synth.mlp_flat(m), n_hidden, f) == 0.5


def test_random_network_vs_matmul():
    m = synth.xavier_mlp()
    rng = np.random.default_rng(5)
    for _ in range(20):
        f = rng.normal(size=NF)
        h = np.maximum(m["W"][0] @ f + m["b"][0], 0)
        h = np.maximum(m["W"][1] @ h + m["b"][1], 0)
        z = (m["W"][2] @ h + m["b"][2])[0]
        assert abs(oracle.mlp_forward(synth.mlp_flat(m), 2, f) - 1 / (1 + math.exp(-z))) < 1e-14


@pytest.mark.parametrize("q", [-1.0, 1.0])
@pytest.mark.parametrize("pt,eta,phi", [(1.2, 0.25, 0.6), (6.0, -0.5, -2.4)])
def test_features_of_a_noiseless_helix(geom_toy, cuts, q, pt, eta, phi):
    e = synth.muon_event(geom_toy, [pt], [eta], [phi], [q], sigma=0.0)
    r = oracle.run_event(geom_toy, e, cuts, synth.mlp_flat(synth.xavier_mlp()), 2)
    m = truth.match_particle(r.t5_hits(), e.pid)
    assert (m == 0).sum() >= 1
    R = pt / synth.K_FIELD
    for i in np.nonzero(m == 0)[0]:
        f = r.t5_feat[i]
        hits = r.t5_hits()[i]
        lo = hits[0::2]
        X, Y, Z = e.x[lo].astype(float), e.y[lo].astype(float), e.z[lo].astype(float)
        lay = [int(geom_toy.layer[e.sensor[h] // 2]) for h in lo]
        assert lay == sorted(lay) and len(set(lay)) == 5
        for j in range(5):
            rj = math.hypot(X[j], Y[j])
            assert abs(f[6 * j + 0] - rj / 100) < 1e-9
            assert abs(f[6 * j + 1] - math.atan2(Y[j], X[j]) / math.pi) < 1e-9
            assert abs(f[6 * j + 2] - Z[j] / 100) < 1e-9
            # pseudorapidity seen from the origin: z/r = sinh(eta) * (arc / chord) of the turn
            psi_j = 2 * math.asin(rj / (2 * R))
            expect_eta = math.asinh(math.sinh(eta) * (psi_j / 2) / math.sin(psi_j / 2))
            assert abs(f[6 * j + 3] * 2.5 - expect_eta) < 1e-5
            assert abs(f[6 * j + 4] * 11 - lay[j]) < 1e-12
            # MD curvature estimate: the chord L->U of a circle through the origin makes
            # an angle with sin = rU/(2R) to the radius of L, so 2*sin/rL = (1/R) (rU/rL)
            up = hits[2 * j + 1]
            rU = math.hypot(float(e.x[up]), float(e.y[up]))
            assert abs(f[6 * j + 5] / 100 + q / R * rU / rj) < 1e-3 / R
        for a, b in ((30, 31), (32, 33)):
            assert abs(f[a] - math.log10(pt)) < 2e-3
            assert abs(f[b] - math.log10(R)) < 2e-3
        assert abs(f[34] - math.log10(pt)) < 2e-3
        assert abs(f[35] * 2.5 - eta) < 1e-3
        # chord P0 -> P4 of a circle points along the tangent at the mid turning angle
        psi = [2 * math.asin(math.hypot(X[j], Y[j]) / (2 * R)) for j in (0, 4)]
        chord_dir = phi - q * 0.5 * (psi[0] + psi[1])
        d = (f[36] * math.pi - chord_dir + math.pi) % (2 * math.pi) - math.pi
        assert abs(d) < 1e-3
        assert abs(f[37] - math.log10(R)) < 2e-3


def test_selection_uses_working_point(geom_toy, cuts):
    e = synth.toy_event(geom_toy, 2)
    m = synth.xavier_mlp()
    r = oracle.run_event(geom_toy, e, cuts, synth.mlp_flat(m), 2)
    assert r.counts["t5"] > 0
    assert np.array_equal(r.t5_sel.astype(bool), r.t5_score >= float(cuts["wp"]))
    for i in range(min(5, r.counts["t5"])):
        assert abs(oracle.mlp_forward(synth.mlp_flat(m), 2, r.t5_feat[i]) - r.t5_score[i]) == 0.0
