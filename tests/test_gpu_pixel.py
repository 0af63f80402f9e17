"""GPU parity of the pixel-seed steps (Table 1 steps 5-8): the track candidates of
lst_match_pixel_seeds, as (type, seed index, object hit tuple), equal the oracle's exactly
(integer work; the matching decisions are FP32 comparisons of the same expression trees and
the one-to-one preference has a total order that does not depend on storage order)."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PC = synth.default_pixel_cuts()


def _cuts():
    c = synth.default_cuts()
    c["wp"] = np.float32(0.0)        # every T5 selected: the track candidates are the deduplicated T5s
    return c


def _gpu_tuples(ev, rows):
    t5 = ev.candidates(lst.LST_T5)[0]
    t3 = ev.candidates(lst.LST_T3)
    out = []
    for typ, p, o in rows.tolist():
        h = t5[o].tolist() if typ in (5, 6) else t3[o].tolist() if typ == 7 else []
        out.append((typ, p, *(h + [-1] * (10 - len(h)))))
    return sorted(out)


def _dev(e):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (e.x, e.y, e.z, e.sensor)]


@pytest.fixture(scope="module")
def ctx(geom_full):
    c = lst.Context(0, max_events=4)
    c.load_geometry(geom_full, _cuts(), synth.mlp_flat(synth.xavier_mlp()), 2)
    yield c
    c.close()


@pytest.mark.parametrize("pileup,index", [(20, 0), (60, 1), (200, 2)])
def test_pixel_candidates_equal_the_oracle(ctx, geom_full, pileup, index):
    e = synth.pileup_event(geom_full, index, pileup=pileup, mean_per_vertex=96)
    s = synth.pixel_seeds(e)
    ref = oracle.run_event(geom_full, e, _cuts(), synth.mlp_flat(synth.xavier_mlp()), 2, pls=s.hits, pcuts=PC)
    ev = ctx.run_event(*_dev(e))
    for seeds in (s.hits, torch.from_numpy(s.hits).cuda()):      # host and device seeds
        cnt = ev.match_pixel_seeds(seeds, PC)
        rows = ev.pixel_candidates()
        got = _gpu_tuples(ev, rows)
        exp = sorted(ref.pixel_tcs())
        assert len(got) == len(exp) == cnt["n_rows"]
        assert got == exp
        ty = rows[:, 0]
        assert [cnt["n_pt5"], cnt["n_t5"], cnt["n_pt3"], cnt["n_pls"]] == [int((ty == k).sum()) for k in (5, 6, 7, 8)]
        assert cnt["n_pt5"] > 0.9 * int(ref.t5_tc.sum())
    print(f"PU{pileup}: {s.n} seeds, {cnt}")
    ev.release()


def test_pixel_without_seeds_and_after_a_batch(ctx, geom_full):
    e = synth.pileup_event(geom_full, 3, pileup=10, mean_per_vertex=96)
    s = synth.pixel_seeds(e)
    hs = ctx.run_batch([_dev(e), _dev(e)])
    assert all(h.counts()["status"] == lst.LST_OK for h in hs)
    # no seeds: every track-candidate T5 stays a T5
    cnt = hs[0].match_pixel_seeds(np.zeros((0, 4, 3), np.float32), PC)
    tc = hs[0].counts()["tc"]
    assert cnt["n_t5"] == cnt["n_rows"] == tc and cnt["n_pt5"] == cnt["n_pt3"] == cnt["n_pls"] == 0
    # seeds on the batched event equal the oracle
    ref = oracle.run_event(geom_full, e, _cuts(), synth.mlp_flat(synth.xavier_mlp()), 2, pls=s.hits, pcuts=PC)
    hs[1].match_pixel_seeds(s.hits, PC)
    assert _gpu_tuples(hs[1], hs[1].pixel_candidates()) == sorted(ref.pixel_tcs())
    for h in hs:
        h.release()
    # a released event has no pixel candidates
    ev = ctx.run_event(*_dev(e))
    with pytest.raises(lst.LstError) as ei:
        ev.pixel_candidates()
    assert ei.value.status == lst.LST_ERR_NOT_READY
    ev.release()


def test_pixel_batch_equals_the_oracle(ctx, geom_full):
    """lst_match_pixel_seeds_batch over a batch of events of uneven size (one without seeds)
    gives each event the oracle's track candidates, as a single call would; counts per event."""
    ev_in = [synth.pileup_event(geom_full, 20 + k, pileup=pu, mean_per_vertex=96) for k, pu in enumerate((60, 10, 120))]
    seeds = [synth.pixel_seeds(e) for e in ev_in]
    hs = ctx.run_batch([_dev(e) for e in ev_in])
    assert all(h.counts()["status"] == lst.LST_OK for h in hs)
    seed_arrays = [seeds[0].hits, np.zeros((0, 4, 3), np.float32), torch.from_numpy(seeds[2].hits).cuda()]
    cnts = ctx.match_pixel_seeds_batch(hs, seed_arrays, PC)
    for k, (e, h, cnt) in enumerate(zip(ev_in, hs, cnts)):
        sd = seeds[k].hits if k != 1 else np.zeros((0, 4, 3), np.float32)
        ref = oracle.run_event(geom_full, e, _cuts(), synth.mlp_flat(synth.xavier_mlp()), 2, pls=sd, pcuts=PC)
        got = _gpu_tuples(h, h.pixel_candidates())
        assert got == sorted(ref.pixel_tcs())
        assert cnt["n_rows"] == len(got)
        if k == 1:
            assert cnt["n_pt5"] == cnt["n_pt3"] == cnt["n_pls"] == 0 and cnt["rounds_pt5"] == 0
        else:
            assert cnt["n_pt5"] > 0 and cnt["rounds_pt5"] >= 2
    # the same event twice is an argument error
    with pytest.raises(lst.LstError) as ei:
        ctx.match_pixel_seeds_batch([hs[0], hs[0]], [seeds[0].hits, seeds[0].hits], PC)
    assert ei.value.status == lst.LST_ERR_ARG
    for h in hs:
        h.release()
