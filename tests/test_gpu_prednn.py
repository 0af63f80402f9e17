"""GPU parity of the pre-DNN mode (the circle-fit chi2 selection of Section 2 in place of
the T5-DNN) and of the track candidates built from the selected T5s: T5 and track-
candidate sets bit-identical to the oracle (every decision is FP32 with the same
expression tree on both sides), every T5 selected, counts equal."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def canon(a):
    return a[np.lexsort(a.T[::-1])] if len(a) else a


def dev(e):
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in (e.x, e.y, e.z, e.sensor)]


def check(ev, ref):
    c = ev.counts()
    assert c["status"] == lst.LST_OK
    hits, _, sel = ev.candidates(lst.LST_T5)
    assert np.array_equal(canon(hits), canon(ref.t5_hits()))
    assert sel.all() and c["selected"] == c["t5"]
    tc, _, tsel = ev.candidates(lst.LST_TC)
    assert c["tc"] == len(tc) == int(ref.t5_tc.sum()) > 0
    assert np.array_equal(canon(tc), canon(ref.tc_hits()))
    assert list(c["pairs"]) == list(ref.pairs)
    return c


@pytest.fixture(scope="module")
def model():
    return synth.mlp_flat(synth.xavier_mlp()), 2


@pytest.mark.parametrize("chi2_max", [5.0, 20.0])
@pytest.mark.parametrize("precision", [lst.LST_FP32, lst.LST_BF16X3])
def test_pre_dnn_mode_pu200(geom_full, model, chi2_max, precision):
    cuts = synth.pre_dnn_cuts(chi2_max)
    e = synth.pileup_event(geom_full, 103, pileup=200, mean_per_vertex=96, config=3)
    ref = oracle.run_event(geom_full, e, cuts, *model)
    c = lst.Context(0, max_events=2, precision=precision)
    c.load_geometry(geom_full, cuts, *model)
    ev = c.run_event(*dev(e))
    cnt = check(ev, ref)
    print(f"pre-DNN chi2<={chi2_max}: {cnt['t5']} T5, {cnt['tc']} track candidates")
    ev.release()
    c.close()


def test_chi2_with_the_standard_cut_set_and_batches(geom_full, model):
    """The chi2 cut on top of the standard tolerances, on events of uneven size, single
    and batched (graph) launches."""
    cuts = synth.default_cuts()
    cuts["t5_chi2_max"] = np.float32(8.0)
    c = lst.Context(0, max_events=8)
    c.load_geometry(geom_full, cuts, *model)
    evs = [synth.pileup_event(geom_full, i, pileup=pu, mean_per_vertex=96, config=4)
           for i, pu in enumerate((30, 170, 5, 90))]
    refs = [oracle.run_event(geom_full, e, cuts, *model) for e in evs]
    for e, r in zip(evs, refs):
        ev = c.run_event(*dev(e))
        check(ev, r)
        ev.release()
    for _ in range(2):
        hs = c.run_batch([dev(e) for e in evs])
        for h, r in zip(hs, refs):
            check(h, r)
            h.release()
    c.close()


def test_track_candidates_to_device_buffers(geom_full, model):
    cuts = synth.pre_dnn_cuts(20.0)
    e = synth.pileup_event(geom_full, 104, pileup=60, mean_per_vertex=96, config=3)
    c = lst.Context(0, max_events=2)
    c.load_geometry(geom_full, cuts, *model)
    ev = c.run_event(*dev(e))
    host, hs, hsel = ev.candidates(lst.LST_TC)
    n = len(host)
    d_out = torch.zeros((n, 10), dtype=torch.int32, device="cuda")
    d_sc = torch.zeros(n, dtype=torch.float32, device="cuda")
    d_sel = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ev.candidates(lst.LST_TC, d_out, d_sc, d_sel)
    torch.cuda.synchronize()
    assert np.array_equal(canon(d_out.cpu().numpy()), canon(host))
    assert np.array_equal(np.sort(d_sc.cpu().numpy()), np.sort(hs))
    ev.release()
    c.close()
