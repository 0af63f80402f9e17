"""GPU parity: the CUDA library (through the C-ABI) against the CPU oracle.

Bar: MD/LS/T3/T5 candidate sets bit-identical after canonical sorting (FP32 cut
arithmetic is the same expression tree on both sides); T5-DNN scores within 1e-6 of the
FP64 oracle; selection flags equal except where the oracle score lies within 1e-5 of the
working point."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCORE_TOL = 1e-6
WP_BAND = 1e-5
KINDS = ((lst.LST_MD, "md_hits"), (lst.LST_LS, "ls_hits"), (lst.LST_T3, "t3_hits"), (lst.LST_T5, "t5_hits"))


from lst_parity import canon_order, expected_tc, near_boundary


def dev(e):
    d = torch.device("cuda:0")
    return [torch.from_numpy(np.ascontiguousarray(a)).to(d) for a in (e.x, e.y, e.z, e.sensor)]


def compare(ev, ref, wp, check_features=False):
    for kind, name in KINDS:
        got = ev.candidates(kind)
        if kind == lst.LST_T5:
            got, score, sel = got
        exp = getattr(ref, name)()
        assert got.shape == exp.shape, (name, got.shape, exp.shape)
        og, oe = canon_order(got), canon_order(exp)
        assert np.array_equal(got[og], exp[oe]), name
    c = ev.counts()
    assert list(c["pairs"]) == list(ref.pairs), (c["pairs"], ref.pairs)
    if len(exp):
        s_ref = ref.t5_score[oe]
        s_got = score[og].astype(np.float64)
        err = np.max(np.abs(s_got - s_ref))
        assert err <= SCORE_TOL, err
        far = np.abs(s_ref - wp) >= WP_BAND
        assert np.array_equal(sel[og][far].astype(bool), (s_ref >= wp)[far])
        if check_features:
            f = ev.features()[og].astype(np.float64)
            df = np.abs(f - ref.t5_feat[oe])
            assert np.max(df) <= 4e-6, (np.max(df), np.unravel_index(np.argmax(df), df.shape))
        # track candidates: the duplicate removal is exact (FP32 chi2 ranks); compared on
        # every event against the oracle's removal run on the GPU's own selection flags
        tc = ev.candidates(lst.LST_TC)[0]
        exp_tc = expected_tc(ref, sel, og, oe)
        assert c["tc"] == len(tc) == len(exp_tc)
        assert np.array_equal(tc[canon_order(tc)], exp_tc[canon_order(exp_tc)])
        if np.array_equal(sel[og], ref.t5_sel[oe]):
            assert len(tc) == int(ref.t5_tc.sum())
    near_boundary(ref)
    return c


@pytest.fixture(scope="module")
def model():
    return synth.mlp_flat(synth.xavier_mlp()), 2


@pytest.fixture(scope="module")
def ctx_toy(geom_toy, cuts, model):
    c = lst.Context(0, max_events=8)
    c.load_geometry(geom_toy, cuts, *model)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_full(geom_full, cuts, model):
    c = lst.Context(0, max_events=16)
    c.load_geometry(geom_full, cuts, *model)
    yield c
    c.close()


@pytest.mark.parametrize("index", [0, 1, 2])
def test_toy_parity(ctx_toy, geom_toy, cuts, model, index):
    e = synth.toy_event(geom_toy, index)
    ref = oracle.run_event(geom_toy, e, cuts, *model)
    ev = ctx_toy.run_event(*dev(e))
    c = compare(ev, ref, float(cuts["wp"]), check_features=True)
    assert c["t5"] == ref.counts["t5"] > 0
    ev.release()


@pytest.mark.parametrize("pileup,index", [(20, 0), (60, 1)])
def test_pileup_slice_parity(ctx_full, geom_full, cuts, model, pileup, index):
    e = synth.pileup_event(geom_full, index, pileup=pileup, mean_per_vertex=96)
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = ctx_full.run_event(*dev(e))
    compare(ev, ref, float(cuts["wp"]), check_features=True)
    ev.release()


def test_pu200_full_parity(ctx_full, geom_full, cuts, model):
    e = synth.pileup_event(geom_full, 0, pileup=200, mean_per_vertex=96)
    assert e.n_hits > 200_000
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = ctx_full.run_event(*dev(e))
    c = compare(ev, ref, float(cuts["wp"]), check_features=True)
    assert c["ls"] > 500_000
    ev.release()


def test_empty_and_degenerate_events(ctx_full, geom_full, cuts, model):
    empty = synth.Event(x=np.zeros(0, np.float32), y=np.zeros(0, np.float32), z=np.zeros(0, np.float32),
                        sensor=np.zeros(0, np.int32), pid=np.zeros(0, np.int32), particles={})
    ev = ctx_full.run_event(*dev(empty))
    c = ev.counts()
    assert c["md"] == c["ls"] == c["t3"] == c["t5"] == 0 and c["status"] == lst.LST_OK
    ev.release()
    # a single track whose hits are all in lower sensors: no MD at all
    e = synth.muon_event(geom_full, [2.0], [0.3], [0.1], [1.0], sigma=0.0)
    keep = e.sensor % 2 == 0
    lo = synth.Event(x=e.x[keep], y=e.y[keep], z=e.z[keep], sensor=e.sensor[keep], pid=e.pid[keep], particles={})
    ev = ctx_full.run_event(*dev(lo))
    assert ev.counts()["md"] == 0
    ev.release()
    # one noiseless track
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = ctx_full.run_event(*dev(e))
    compare(ev, ref, float(cuts["wp"]))
    ev.release()


def test_invalid_hits_report_input_error(ctx_full, geom_full, cuts, model):
    e = synth.pileup_event(geom_full, 3, pileup=5, mean_per_vertex=96)
    for mutate in ("sensor", "nan"):
        x, s = e.x.copy(), e.sensor.copy()
        if mutate == "sensor":
            s[7] = geom_full.n_sensor + 3
        else:
            x[11] = np.nan
        bad = synth.Event(x=x, y=e.y, z=e.z, sensor=s, pid=e.pid, particles={})
        ev = ctx_full.run_event(*dev(bad))
        assert ev.status == lst.LST_ERR_INPUT
        ev.release()
    # the context stays usable
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = ctx_full.run_event(*dev(e))
    compare(ev, ref, float(cuts["wp"]))
    ev.release()


def test_overflow_regrows_to_exact_result(geom_full, cuts, model):
    c = lst.Context(0, max_events=2, md_per_hit=0.001, ls_per_md=0.01, t3_per_md=0.01, t5_per_md=0.01)
    c.load_geometry(geom_full, cuts, *model)
    e = synth.pileup_event(geom_full, 4, pileup=30, mean_per_vertex=96)
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = c.run_event(*dev(e))
    compare(ev, ref, float(cuts["wp"]))
    ev.release()
    c.close()


def test_batch_with_overflowing_events(geom_full, cuts, model):
    """A batch in which the large events overflow their T3 buffer and the small ones do not:
    the small ones must still be exact (the stage's work split between CTAs must not change
    when an event overflows mid-kernel), and re-running the large ones regrows to exact."""
    c = lst.Context(0, max_events=8, t3_per_md=0.01, t5_per_md=0.01)
    c.load_geometry(geom_full, cuts, *model)
    evs = [synth.pileup_event(geom_full, 50 + i, pileup=pu, mean_per_vertex=96, config=4)
           for i, pu in enumerate((1, 200, 1, 120, 2))]
    refs = [oracle.run_event(geom_full, e, cuts, *model) for e in evs]
    hs = c.run_batch([dev(e) for e in evs])
    st = [h.counts()["status"] for h in hs]
    assert st[1] == lst.LST_ERR_CAPACITY and st[3] == lst.LST_ERR_CAPACITY
    for k in (0, 2, 4):
        assert st[k] == lst.LST_OK
        compare(hs[k], refs[k], float(cuts["wp"]))
    for h in hs:
        h.release()
    for k in (1, 3):
        ev = c.run_event(*dev(evs[k]))
        compare(ev, refs[k], float(cuts["wp"]))
        ev.release()
    c.close()


def test_list_overflow_paths(geom_full, cuts, model):
    """Tiny candidate lists force the re-evaluation paths of the MD and LS kernels, odd CTA
    sizes change every work decomposition; results must not change."""
    c = lst.Context(0, max_events=2)
    c.load_geometry(geom_full, cuts, *model)
    c.set_launch(md_buf=1, ls_list=2, md_threads=64, ls_threads=64, t3_threads=96, t5_threads=160)
    e = synth.pileup_event(geom_full, 5, pileup=40, mean_per_vertex=96)
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = c.run_event(*dev(e))
    compare(ev, ref, float(cuts["wp"]))
    ev.release()
    c.close()


def test_batches_in_flight(geom_full, cuts, model):
    """Four batches launched without reading anything in between: three lanes hold the first
    three, the fourth waits for the first lane's batch and reuses that lane; every event of
    every batch equals the oracle."""
    c = lst.Context(0, max_events=16)
    c.load_geometry(geom_full, cuts, *model)
    evs = [synth.pileup_event(geom_full, 80 + i, pileup=pu, mean_per_vertex=96)
           for i, pu in enumerate((20, 3, 30, 10, 25, 5, 15, 35))]
    refs = [oracle.run_event(geom_full, e, cuts, *model) for e in evs]
    inputs = [dev(e) for e in evs]
    batches = [c.run_batch(inputs[2 * b:2 * b + 2]) for b in range(4)]
    for b, hs in enumerate(batches):
        for k, h in enumerate(hs):
            assert h.counts()["status"] == lst.LST_OK
            compare(h, refs[2 * b + k], float(cuts["wp"]))
            h.release()
    c.close()


def test_batch_equals_single_and_graph_replay(ctx_full, geom_full, cuts, model):
    evs = [synth.pileup_event(geom_full, i, pileup=pu, mean_per_vertex=96, config=4)
           for i, pu in enumerate((50, 250, 120, 7, 180, 90))]
    inputs = [dev(e) for e in evs]
    singles = []
    for t in inputs:
        ev = ctx_full.run_event(*t)
        singles.append({k: np.sort(ev.candidates(k)[0] if k == lst.LST_T5 else ev.candidates(k), axis=0)
                        for k, _ in KINDS})
        ev.release()
    for rep in range(3):   # first run captures the graph, later runs replay it
        handles = ctx_full.run_batch(inputs)
        for h, s, e in zip(handles, singles, evs):
            assert h.counts()["status"] == lst.LST_OK
            for k, _ in KINDS:
                got = h.candidates(k)
                got = got[0] if k == lst.LST_T5 else got
                assert np.array_equal(np.sort(got, axis=0), s[k])
            h.release()
    # one batched event also against the oracle
    ref = oracle.run_event(geom_full, evs[1], cuts, *model)
    h = ctx_full.run_batch(inputs[1:2])[0]
    compare(h, ref, float(cuts["wp"]))
    h.release()


def test_batched_export_equals_per_event_export(ctx_full, geom_full):
    evs = [synth.pileup_event(geom_full, i, pileup=pu, mean_per_vertex=96, config=4)
           for i, pu in enumerate((40, 5, 0, 90))]
    hs = ctx_full.run_batch([dev(e) for e in evs])
    for kind in (lst.LST_LS, lst.LST_T5, lst.LST_TC):
        out, score, sel, offs = ctx_full.candidates_batch(hs, kind)
        assert offs[0] == 0 and len(out) == offs[-1]
        d_out = torch.zeros((int(offs[-1]) + 7, lst.WIDTH[kind]), dtype=torch.int32, device="cuda")
        _, _, _, offs2 = ctx_full.candidates_batch(hs, kind, d_out)
        assert np.array_equal(offs, offs2)
        dev_rows = d_out.cpu().numpy()
        for i, h in enumerate(hs):
            single = h.candidates(kind)
            single = single[0] if kind in (lst.LST_T5, lst.LST_TC) else single
            rows = out[offs[i]:offs[i + 1]]
            assert np.array_equal(np.sort(rows, axis=0), np.sort(single, axis=0))
            if kind != lst.LST_TC:   # the track-candidate gather has no fixed order
                assert np.array_equal(dev_rows[offs[i]:offs[i + 1]], rows)
            else:
                assert np.array_equal(np.sort(dev_rows[offs[i]:offs[i + 1]], axis=0), np.sort(rows, axis=0))
    for h in hs:
        h.release()


def test_host_inputs_match_device_inputs(ctx_full, geom_full, cuts, model):
    e = synth.pileup_event(geom_full, 6, pileup=25, mean_per_vertex=96)
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = ctx_full.run_event(e.x, e.y, e.z, e.sensor)
    compare(ev, ref, float(cuts["wp"]))
    ev.release()


def test_score_t5_standalone_fp32(ctx_full, model):
    rng = np.random.default_rng(11)
    f = rng.normal(0, 1, (5000, 38)).astype(np.float32)
    d = torch.from_numpy(f).cuda()
    out = torch.empty(5000, dtype=torch.float32, device="cuda")
    ctx_full.score_t5(d, out, lst.LST_FP32)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    exp = np.array([oracle.mlp_forward(model[0], 2, f[i].astype(np.float64)) for i in range(0, 5000, 7)])
    assert np.max(np.abs(got[::7] - exp)) <= SCORE_TOL


# --------------------------------------------------------------------------- BF16 tensor cores
BF16_TOL = 2e-2   # stated bound of the BF16 score (BF16 operands, FP32 accumulation) vs FP64


def test_score_t5_standalone_bf16(ctx_full, model):
    rng = np.random.default_rng(12)
    f = rng.normal(0, 1, (4099, 38)).astype(np.float32)   # ragged last tile of 128 rows
    d = torch.from_numpy(f).cuda()
    out32 = torch.empty(4099, dtype=torch.float32, device="cuda")
    out16 = torch.empty(4099, dtype=torch.float32, device="cuda")
    ctx_full.score_t5(d, out32, lst.LST_FP32)
    ctx_full.score_t5(d, out16, lst.LST_BF16)
    torch.cuda.synchronize()
    assert lst.load_library().lst_device_errors(ctx_full.h) == lst.LST_OK
    a, b = out32.cpu().numpy().astype(np.float64), out16.cpu().numpy().astype(np.float64)
    exp = np.array([oracle.mlp_forward(model[0], 2, f[i].astype(np.float64)) for i in range(0, 4099, 5)])
    err = np.max(np.abs(b[::5] - exp))
    print(f"bf16 standalone max|dscore| vs fp64 = {err:.3e}")
    assert err <= BF16_TOL
    assert np.max(np.abs(a[::5] - exp)) <= SCORE_TOL


def test_bf16_event_path(geom_full, cuts, model):
    c = lst.Context(0, max_events=4, precision=lst.LST_BF16)
    c.load_geometry(geom_full, cuts, *model)
    e = synth.pileup_event(geom_full, 9, pileup=120, mean_per_vertex=96)
    ref = oracle.run_event(geom_full, e, cuts, *model)
    ev = c.run_event(*dev(e))
    hits, score, sel = ev.candidates(lst.LST_T5)
    exp = ref.t5_hits()
    og, oe = canon_order(hits), canon_order(exp)
    assert np.array_equal(hits[og], exp[oe])          # the cuts are FP32 in both precisions
    err = np.max(np.abs(score[og].astype(np.float64) - ref.t5_score[oe]))
    flips = int(np.sum(sel[og].astype(bool) != (ref.t5_score[oe] >= float(cuts["wp"]))))
    print(f"bf16 event path: {len(hits)} T5, max|dscore| = {err:.3e}, selection flips = {flips}")
    assert err <= BF16_TOL
    # a flip needs the FP64 score within the error of the working point
    near = np.abs(ref.t5_score[oe] - float(cuts["wp"])) <= err
    assert np.all((sel[og].astype(bool) == (ref.t5_score[oe] >= float(cuts["wp"]))) | near)
    ev.release()
    # batched BF16 (graph) path gives the same scores as the single-event BF16 path
    h = c.run_batch([dev(e)])[0]
    hb, sb, _ = h.candidates(lst.LST_T5)
    ob = canon_order(hb)
    assert np.array_equal(hb[ob], hits[og]) and np.array_equal(sb[ob], score[og])
    h.release()
    c.close()
