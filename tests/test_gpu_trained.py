"""GPU parity with the project-trained T5-DNNs (1 to 4 hidden layers of 32) on the open-cut
set they were trained with.

The trained networks are ill-conditioned in their log-curvature inputs (the score moves by
up to ~200 per unit of those features), so a single FP32 rounding of a feature already
moves the score by ~1e-5: the 1e-6 score bar of the FP32 path (seeded random weights)
cannot hold here and is replaced by the checks below.
  * candidate sets bit-identical to the oracle (the cuts do not involve the network);
  * features within 4e-6 of the oracle's FP64 features;
  * FP32 score against the FP64 network evaluated on the GPU's own FP32 features, within
    the a priori rounding bound of FP32 dot products (|fl(x.y) - x.y| <= gamma_n |x|.|y|,
    gamma_n = n u / (1 - n u), u = 2^-24; Higham, Accuracy and Stability of Numerical
    Algorithms, Section 3.1) propagated through the layers, times the sigmoid's slope 1/4;
  * FP32 and split-BF16 (LST_BF16X3) scores against the FP64 oracle within the stated
    bounds FP32_TRAINED_TOL and BF16X3_TOL, selection flips only where the FP64 score lies
    within the observed error of the working point;
  * plain BF16 is reported (error, flips) but has no bound for these networks;
  * track candidates equal the oracle's duplicate removal run on the GPU's own selection
    flags, at every precision."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import lst, model_store, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FEATURE_TOL = 4e-6
FP32_TRAINED_TOL = 2e-3
BF16X3_TOL = 1e-2
U32 = 2.0 ** -24


from lst_parity import canon_order, expected_tc


def dev(e):
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in (e.x, e.y, e.z, e.sensor)]


def layers(flat, n_hidden):
    out, o = [], 0
    for l in range(n_hidden):
        k = 38 if l == 0 else 32
        W = flat[o:o + 32 * k].reshape(32, k)
        o += 32 * k
        out.append((W, flat[o:o + 32]))
        o += 32
    out.append((flat[o:o + 32].reshape(1, 32), flat[o + 32:o + 33]))
    return out


def fp32_bound(flat, n_hidden, F):
    """Per-row bound on |FP32 network score - exact score| for FP32 inputs F (exact values)."""
    h = F.astype(np.float64)
    e = np.zeros_like(h)
    gam = lambda n: n * U32 / (1 - n * U32)
    net = layers(np.asarray(flat, np.float32).astype(np.float64), n_hidden)
    for i, (W, b) in enumerate(net):
        aW = np.abs(W)
        s = h @ W.T + b
        mag = np.abs(h) @ aW.T + np.abs(b) + e @ aW.T
        e = e @ aW.T + gam(W.shape[1] + 1) * mag
        h = np.maximum(s, 0.0) if i + 1 < len(net) else s
    return 0.25 * e[:, 0] + 1e-6       # sigmoid slope <= 1/4; the exp and divide add < 1e-6


@pytest.fixture(scope="module")
def event(geom_full):
    return synth.pileup_event(geom_full, 101, pileup=200, mean_per_vertex=96, config=3)


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_trained_network_parity(geom_full, event, depth):
    w = model_store.load(f"{model_store.WEIGHTS_DIR}/t5dnn_{depth}x32.npz")
    cuts = synth.open_cuts()
    cuts["wp"] = np.float32(w["wp"])
    wp = float(cuts["wp"])
    ref = oracle.run_event(geom_full, event, cuts, w["flat"], depth)
    exp = ref.t5_hits()
    oe = canon_order(exp)
    s_ref = ref.t5_score[oe]
    for prec in (lst.LST_FP32, lst.LST_BF16X3, lst.LST_BF16):
        c = lst.Context(0, max_events=2, precision=prec)
        c.load_geometry(geom_full, cuts, w["flat"], depth)
        ev = c.run_event(*dev(event))
        assert ev.status == lst.LST_OK
        hits, score, sel = ev.candidates(lst.LST_T5)
        og = canon_order(hits)
        assert np.array_equal(hits[og], exp[oe])
        s_got = score[og].astype(np.float64)
        err = float(np.max(np.abs(s_got - s_ref)))
        flips = int(np.sum(sel[og].astype(bool) != (s_ref >= wp)))
        print(f"{depth}x32 precision {prec}: {len(hits)} T5, max|dscore| vs FP64 {err:.3e}, flips {flips}")
        if prec == lst.LST_FP32:
            f = ev.features()[og]
            df = float(np.max(np.abs(f.astype(np.float64) - ref.t5_feat[oe])))
            assert df <= FEATURE_TOL, df
            step = max(1, len(f) // 4000)          # the FP64 network on the GPU's own features
            exact = np.array([oracle.mlp_forward(w["flat"], depth, f[i].astype(np.float64))
                              for i in range(0, len(f), step)])
            bound = fp32_bound(w["flat"], depth, f[::step])
            d = np.abs(s_got[::step] - exact)
            print(f"   features max|df| {df:.2e}; FP32 arithmetic max|ds| {d.max():.2e}, "
                  f"min bound/|ds| {np.min(bound / np.maximum(d, 1e-30)):.1f}")
            assert np.all(d <= bound)
            assert err <= FP32_TRAINED_TOL
        if prec == lst.LST_BF16X3:
            assert err <= BF16X3_TOL
        if prec != lst.LST_BF16:
            near = np.abs(s_ref - wp) <= max(err, 1e-5)
            assert np.all((sel[og].astype(bool) == (s_ref >= wp)) | near)
        # track candidates, every precision (plain BF16 included, with its many flips):
        # the oracle's duplicate removal on the GPU's own selection flags
        tc = ev.candidates(lst.LST_TC)[0]
        exp_tc = expected_tc(ref, sel, og, oe)
        assert np.array_equal(tc[canon_order(tc)], exp_tc[canon_order(exp_tc)])
        ev.release()
        c.close()


def test_bf16x3_standalone_matches_event_path(geom_full, event):
    """lst_score_t5 in split mode on the event's features gives the fused event path's scores."""
    w = model_store.load(f"{model_store.WEIGHTS_DIR}/t5dnn_2x32.npz")
    cuts = synth.open_cuts()
    c = lst.Context(0, max_events=2, precision=lst.LST_BF16X3)
    c.load_geometry(geom_full, cuts, w["flat"], 2)
    ev = c.run_event(*dev(event))
    _, score, _ = ev.candidates(lst.LST_T5)
    f = torch.from_numpy(ev.features()).cuda()
    out = torch.empty(len(f), dtype=torch.float32, device="cuda")
    c.score_t5(f, out, lst.LST_BF16X3)
    torch.cuda.synchronize()
    assert lst.load_library().lst_device_errors(c.h) == lst.LST_OK
    assert np.array_equal(out.cpu().numpy(), score)
    ev.release()
    c.close()
