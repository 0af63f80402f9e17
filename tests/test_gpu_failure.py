"""GPU failure handling without a fault: the tensor-core score kernels wait for their MMAs
with an iteration limit. With the test aid that makes them issue no MMA, nothing ever
arrives on that wait; it runs out, the events report LST_ERR_TIMEOUT, lst_device_errors
returns it once, and the same context then produces correct results again."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def canon(a):
    return a[np.lexsort(a.T[::-1])] if len(a) else a


@pytest.mark.parametrize("precision", [lst.LST_BF16, lst.LST_BF16X3])
def test_bounded_mma_wait_times_out_and_recovers(geom_full, cuts, precision):
    w = synth.mlp_flat(synth.xavier_mlp())
    e = synth.pileup_event(geom_full, 11, pileup=20, mean_per_vertex=96)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (e.x, e.y, e.z, e.sensor)]
    c = lst.Context(0, max_events=4, precision=precision)
    c.load_geometry(geom_full, cuts, w, 2)
    c.set_wait_limit(2000)
    c.test_skip_mma(True)
    ev = c.run_event(*d)                      # single-event path
    assert ev.status == lst.LST_ERR_TIMEOUT
    ev.release()
    assert c.device_errors() == lst.LST_ERR_TIMEOUT
    assert c.device_errors() == lst.LST_OK   # reported once
    hs = c.run_batch([d, d])                  # batched (graph) path
    assert all(h.counts()["status"] == lst.LST_ERR_TIMEOUT for h in hs)
    for h in hs:
        h.release()
    f = torch.zeros((300, 38), dtype=torch.float32, device="cuda")
    out = torch.zeros(300, dtype=torch.float32, device="cuda")
    c.score_t5(f, out, precision)             # standalone scoring
    assert c.device_errors() == lst.LST_ERR_TIMEOUT
    # back to normal: the context is usable and correct
    c.test_skip_mma(False)
    c.set_wait_limit(1 << 26)
    ev = c.run_event(*d)
    assert ev.status == lst.LST_OK
    hits, score, _ = ev.candidates(lst.LST_T5)
    ref = oracle.run_event(geom_full, e, cuts, w, 2)
    assert np.array_equal(canon(hits), canon(ref.t5_hits()))
    assert np.max(np.abs(np.sort(score.astype(np.float64)) - np.sort(ref.t5_score))) <= 2e-2
    ev.release()
    assert c.device_errors() == lst.LST_OK
    c.close()


def test_injected_allocation_failures_leave_the_context_usable(geom_full, cuts):
    """Host-side allocation-failure injection: the creation and the growth of an event
    slot's buffers, the staging of host inputs and a batch all fail with LST_ERR_NOMEM when
    their allocation is made to fail; no event is produced, and the same calls succeed
    afterwards with oracle-identical candidates."""
    w = synth.mlp_flat(synth.xavier_mlp())
    small = synth.pileup_event(geom_full, 12, pileup=10, mean_per_vertex=96)
    big = synth.pileup_event(geom_full, 13, pileup=60, mean_per_vertex=96)
    dev = lambda e: [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (e.x, e.y, e.z, e.sensor)]
    host = lambda e: [np.ascontiguousarray(a) for a in (e.x, e.y, e.z, e.sensor)]
    refs = {id(e): oracle.run_event(geom_full, e, cuts, w, 2) for e in (small, big)}

    def check(ev, e):
        assert ev.counts()["status"] == lst.LST_OK
        for kind, name in ((lst.LST_MD, "md_hits"), (lst.LST_LS, "ls_hits"), (lst.LST_T5, "t5_hits")):
            got = ev.candidates(kind)
            got = got[0] if isinstance(got, tuple) else got
            assert np.array_equal(canon(got), canon(getattr(refs[id(e)], name)())), name
        ev.release()

    c = lst.Context(0, max_events=4)
    c.load_geometry(geom_full, cuts, w, 2)
    # 1. the first allocation of a slot
    c.test_fail_alloc(1)
    with pytest.raises(lst.LstError) as ei:
        c.run_event(*dev(small))
    assert ei.value.status == lst.LST_ERR_NOMEM and "injected" in str(ei.value)
    check(c.run_event(*dev(small)), small)
    # 2. growth of that slot for a larger event
    c.test_fail_alloc(1)
    with pytest.raises(lst.LstError) as ei:
        c.run_event(*dev(big))
    assert ei.value.status == lst.LST_ERR_NOMEM
    check(c.run_event(*dev(small)), small)       # smaller again: the slot reallocates
    check(c.run_event(*dev(big)), big)
    # 3. staging of host inputs (the slot's buffers exist; the input copy needs memory)
    c.test_fail_alloc(1)
    with pytest.raises(lst.LstError) as ei:
        c.run_event(*host(big))
    assert ei.value.status == lst.LST_ERR_NOMEM
    check(c.run_event(*host(small)), small)
    check(c.run_event(*host(big)), big)
    # 4. a batch whose later slots cannot be allocated
    c.test_fail_alloc(2)
    with pytest.raises(lst.LstError) as ei:
        c.run_batch([dev(big), dev(small), dev(big), dev(big)])
    assert ei.value.status == lst.LST_ERR_NOMEM
    c.test_fail_alloc(0)
    hs = c.run_batch([dev(big), dev(small), dev(big)])
    for h, e in zip(hs, (big, small, big)):
        check(h, e)
    assert c.device_errors() == lst.LST_OK
    c.close()
