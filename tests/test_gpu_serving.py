"""Serving with continuous batching: events submitted one by one while others run on the
GPU give exactly the results they give alone (lst_run_event), and every request finishes."""
import time

import numpy as np
import pytest

from paper_2403_13166_gb300 import lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _overlapping(results):
    """Pairs of requests whose [t_admit, t_done] intervals overlap (both on the GPU side)."""
    r = sorted(results, key=lambda x: x["t_admit"])
    return sum(1 for i in range(len(r)) for j in range(i + 1, len(r)) if r[j]["t_admit"] < r[i]["t_done"])


@pytest.mark.parametrize("precision", [lst.LST_FP32, lst.LST_BF16, lst.LST_BF16X3])
def test_served_results_equal_alone(geom_full, cuts, precision):
    w = synth.mlp_flat(synth.xavier_mlp())
    events = [synth.pileup_event(geom_full, i, pileup=pu, mean_per_vertex=96, config=5)
              for i, pu in enumerate((140, 30, 200, 75, 160, 10, 190, 120, 55, 170, 95, 145))]
    alone = lst.Context(0, max_events=2, precision=precision)
    alone.load_geometry(geom_full, cuts, w, 2)
    ref = []
    for e in events:
        ev = alone.run_event(e.x, e.y, e.z, e.sensor)
        h, s, _ = ev.candidates(lst.LST_T5)
        o = np.lexsort(h.T[::-1])
        ref.append((h[o], s[o]))
        ev.release()
    alone.close()

    ctx = lst.Context(0, max_events=8, precision=precision)
    ctx.load_geometry(geom_full, cuts, w, 2)
    # a small memory budget forces admission to wait for memory as well as slots
    srv = lst.Server(ctx, max_batch=3, lanes=2, mem_budget_bytes=300 << 20, copy_t5=True)
    results = {}
    for k, e in enumerate(events):
        srv.submit(e.x, e.y, e.z, e.sensor, tag=k)          # arrival = now
        time.sleep(0.0005)
        for r in srv.poll():
            results[r["tag"]] = r
    deadline = time.time() + 60
    while len(results) < len(events) and time.time() < deadline:
        for r in srv.poll(wait_ms=50):
            results[r["tag"]] = r
    srv.stop()
    ctx.close()
    assert sorted(results) == list(range(len(events)))
    for k, (h, s) in enumerate(ref):
        r = results[k]
        assert r["status"] == lst.LST_OK
        assert r["t_done"] >= r["t_launch"] >= r["t_admit"] >= r["t_arrival"]
        hh = r.get("t5_hits", np.zeros((0, 10), np.int32))
        o = np.lexsort(hh.T[::-1]) if len(hh) else np.zeros(0, int)
        assert np.array_equal(hh[o], h)
        assert np.array_equal(r["t5_score"][o], s)      # bit-identical: each row scored alone
    assert _overlapping(list(results.values())) > 0   # requests were in flight together


def test_memory_budget_admits_one_event_at_a_time(geom_full, cuts):
    """With a budget below one event's estimated object-buffer memory, an event is only
    admitted when nothing else is in flight; with a large budget they overlap."""
    w = synth.mlp_flat(synth.xavier_mlp())
    events = [synth.pileup_event(geom_full, i, pileup=pu, mean_per_vertex=96, config=5)
              for i, pu in enumerate((150, 60, 180, 90, 120, 30))]
    out = {}
    for budget in (1, 64 << 30):
        ctx = lst.Context(0, max_events=8, precision=lst.LST_BF16X3)
        ctx.load_geometry(geom_full, cuts, w, 2)
        srv = lst.Server(ctx, max_batch=4, lanes=2, mem_budget_bytes=budget, copy_t5=False)
        for k, e in enumerate(events):
            srv.submit(e.x, e.y, e.z, e.sensor, tag=k)
        res = []
        deadline = time.time() + 60
        while len(res) < len(events) and time.time() < deadline:
            res.extend(srv.poll(wait_ms=50))
        srv.stop()
        ctx.close()
        assert len(res) == len(events) and all(r["status"] == lst.LST_OK for r in res)
        out[budget] = _overlapping(res)
    assert out[1] == 0
    assert out[64 << 30] > 0


def test_serve_rejects_bad_config(geom_full, cuts):
    ctx = lst.Context(0, max_events=2)
    ctx.load_geometry(geom_full, cuts)
    with pytest.raises(lst.LstError):
        lst.Server(ctx, max_batch=5)          # more than the context's event slots
    ctx.close()


def test_results_point_into_staging_and_outlive_the_server(geom_full, cuts):
    """Polled results refer to the server's pinned staging (no copy): they hold the same T5
    tuples as the event alone, stay readable after lst_serve_stop until freed, and freeing
    them afterwards (the last one frees the staging) is clean; the staging of freed results
    is reused, so many more batches than stages go through."""
    import ctypes as C
    w = synth.mlp_flat(synth.xavier_mlp())
    events = [synth.pileup_event(geom_full, 40 + i, pileup=pu, mean_per_vertex=96, config=5)
              for i, pu in enumerate((60, 20, 90))]
    alone = lst.Context(0, max_events=2, precision=lst.LST_BF16X3)
    alone.load_geometry(geom_full, cuts, w, 2)
    ref = []
    for e in events:
        ev = alone.run_event(e.x, e.y, e.z, e.sensor)
        h = ev.candidates(lst.LST_T5)[0]
        ref.append(h[np.lexsort(h.T[::-1])])
        ev.release()
    alone.close()

    ctx = lst.Context(0, max_events=4, precision=lst.LST_BF16X3)
    ctx.load_geometry(geom_full, cuts, w, 2)
    # every slot sized at start (slot_hits), as a latency-sensitive server would
    srv = lst.Server(ctx, max_batch=2, lanes=2, mem_budget_bytes=8 << 30, copy_t5=True,
                     slot_hits=int(1.2 * max(len(e.x) for e in events)))
    lib = lst.load_library()
    # many batches through, results freed as they come (the staging is reused)
    for k in range(24):
        e = events[k % 3]
        srv.submit(e.x, e.y, e.z, e.sensor, tag=k)
    got = []
    deadline = time.time() + 60
    while len(got) < 24 and time.time() < deadline:
        got.extend(srv.poll(wait_ms=50))
    assert len(got) == 24 and all(r["status"] == lst.LST_OK for r in got)
    for r in got:
        h = r["t5_hits"]
        assert np.array_equal(h[np.lexsort(h.T[::-1])], ref[r["tag"] % 3])
    # raw results kept past stop
    for k, e in enumerate(events):
        srv.submit(e.x, e.y, e.z, e.sensor, tag=100 + k)
    buf = (lst.lst_serve_result * 8)()
    held = []
    deadline = time.time() + 60
    while len(held) < 3 and time.time() < deadline:
        n = C.c_int32(0)
        assert lib.lst_serve_poll(srv.h, buf, 8, C.byref(n), 50) == lst.LST_OK
        for i in range(n.value):
            r = lst.lst_serve_result()
            C.memmove(C.byref(r), C.byref(buf[i]), C.sizeof(r))
            held.append(r)
    srv.stop()
    ctx.close()
    assert len(held) == 3
    for r in held:
        assert r.status == lst.LST_OK and r.owner
        n5 = r.n_t5
        h = np.ctypeslib.as_array((C.c_int32 * (n5 * 10)).from_address(r.t5_hits)).reshape(n5, 10).copy()
        assert np.array_equal(h[np.lexsort(h.T[::-1])], ref[r.tag - 100])
        assert lib.lst_serve_free_result(C.byref(r)) == lst.LST_OK
        assert not r.owner and not r.t5_hits
