"""The project-trained T5-DNN files (Section 2: 38 features, hidden layers of 32, sigmoid out,
binary cross entropy on truth labels) evaluated by the FP64 oracle on an event none of
them was trained on. CPU only."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import model_store, synth, truth

DEPTHS = (1, 2, 3, 4)


def _load(depth):
    path = f"{model_store.WEIGHTS_DIR}/t5dnn_{depth}x32.npz"
    return model_store.load(path)


def _auc(score, real):
    order = np.argsort(-score, kind="stable")
    r = real[order]
    tp = np.cumsum(r) / max(1, r.sum())
    fp = np.cumsum(~r) / max(1, (~r).sum())
    return float(np.sum(np.diff(np.concatenate([[0.0], fp])) * tp))


@pytest.mark.parametrize("depth", DEPTHS)
def test_weight_file_layout(depth):
    w = _load(depth)
    assert w["n_hidden"] == depth
    # Linear(38,32) + (depth-1) x Linear(32,32) + Linear(32,1), weights and biases
    assert w["flat"].shape == (38 * 32 + 32 + (depth - 1) * (32 * 32 + 32) + 32 + 1,)
    assert np.all(np.isfinite(w["flat"]))
    assert 0.0 < w["wp"] < 1.0
    assert w["meta"]["hidden_layers"] == depth


@pytest.fixture(scope="module")
def held_out():
    """One PU200-like event of the training generator (config 3) with an index outside the
    training range, built with the open-cut set the networks were trained on."""
    g = synth.build_geometry(True)
    e = synth.pileup_event(g, 100, pileup=200, mean_per_vertex=96, config=3)
    cuts = synth.open_cuts()
    ref = oracle.run_event(g, e, cuts, synth.mlp_flat(synth.xavier_mlp()), 2)
    real = truth.t5_labels(ref.t5_hits(), e.pid).astype(bool)
    return ref, real


def test_trained_networks_separate_real_from_fake(held_out):
    ref, real = held_out
    assert len(real) > 50_000 and 0.3 < real.mean() < 0.9      # the sample holds many fakes
    auc = {}
    for depth in DEPTHS:
        w = _load(depth)
        s = np.array([oracle.mlp_forward(w["flat"], depth, f) for f in ref.t5_feat])
        auc[depth] = _auc(s, real)
        eff = float((s[real] >= w["wp"]).mean())
        fake = float((s[~real] >= w["wp"]).mean())
        print(f"{depth}x32: auc {auc[depth]:.4f}  eff {eff:.4f}  fake {fake:.4f}")
        assert eff > 0.9 and fake < 0.2
    assert auc[2] > 0.97
    assert auc[1] < auc[2] < auc[4]           # the depth scan of Section 2: depth helps, less and less
