"""GPU parity in the launch configuration the benchmark times: 64 PU200-like events in one
batched launch per stage (CUDA graph), split-BF16 tensor-core score with the trained 2x32
network, launch shapes from the autotuner. Sampled events against the oracle (candidate
sets bit-identical, scores within the split-BF16 bound, track candidates identical to
the oracle's duplicate removal on the GPU's selection); every event of the batch against
its own single-event run."""
import numpy as np
import pytest

import oracle
from lst_parity import expected_tc, near_boundary
from paper_2403_13166_gb300 import autotune, lst, model_store, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BF16X3_TOL = 1e-2


def canon(a):
    return a[np.lexsort(a.T[::-1])] if len(a) else a


def test_bench_launch_configuration(geom_full, tmp_path):
    w = model_store.load_trained()
    cuts = synth.default_cuts()
    cuts["wp"] = np.float32(w["wp"])
    events = [synth.pileup_event(geom_full, 40_000 + i, pileup=200, mean_per_vertex=96) for i in range(64)]
    d = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (e.x, e.y, e.z, e.sensor)] for e in events]
    ctx = lst.Context(0, max_events=128, precision=lst.LST_BF16X3, use_graphs=1)
    ctx.load_geometry(geom_full, cuts, w["flat"], w["n_hidden"])
    autotune.tune_or_load(ctx, d, path=str(tmp_path / "cache.json"), reps=1)
    for _ in range(2):                        # capture, then replay the graph
        hs = ctx.run_batch(d)
        got = [(canon(h.candidates(lst.LST_T5)[0]), h.counts()) for h in hs]
        for h in hs:
            h.release()
    assert all(c["status"] == lst.LST_OK for _, c in got)
    # every event equals its own single-event run (same context, same precision)
    for k in range(0, 64, 7):
        ev = ctx.run_event(*d[k])
        assert np.array_equal(canon(ev.candidates(lst.LST_T5)[0]), got[k][0])
        assert ev.counts()["tc"] == got[k][1]["tc"]
        ev.release()
    # sampled events against the oracle
    hs = ctx.run_batch(d)
    for k in (0, 31, 63):
        e = events[k]
        ref = oracle.run_event(geom_full, e, cuts, w["flat"], w["n_hidden"])
        hits, score, sel = hs[k].candidates(lst.LST_T5)
        og, oe = np.lexsort(hits.T[::-1]), np.lexsort(ref.t5_hits().T[::-1])
        assert np.array_equal(hits[og], ref.t5_hits()[oe])
        for kind, name in ((lst.LST_MD, "md_hits"), (lst.LST_LS, "ls_hits"), (lst.LST_T3, "t3_hits")):
            assert np.array_equal(canon(hs[k].candidates(kind)), canon(getattr(ref, name)()))
        err = float(np.max(np.abs(score[og].astype(np.float64) - ref.t5_score[oe])))
        assert err <= BF16X3_TOL, err
        tc = hs[k].candidates(lst.LST_TC)[0]
        assert np.array_equal(canon(tc), canon(expected_tc(ref, sel, og, oe)))
        assert list(hs[k].counts()["pairs"]) == list(ref.pairs)
        near_boundary(ref, f"event {k}")
    for h in hs:
        h.release()
    ctx.close()
