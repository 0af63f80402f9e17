"""lst_find_minidoublets_noalloc: the mini-doublet finder for callers that cannot allocate
device memory while they run (for instance code inside a framework that owns all device
memory through its own allocator, or latency-bound loops that cannot absorb the
synchronisation of cudaMalloc/cudaFree). It works in a fixed scratch array compiled into
the library, so its results must equal those of the allocating path (lst_run_event +
lst_get_candidates) exactly, call after call, although every call reuses that array.

Kept in a file that pytest collects last; it passes alone in a fresh process and after
the rest of the suite."""
import numpy as np
import pytest

from paper_2403_13166_gb300 import lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sorted_rows(a):
    a = np.asarray(a)
    return a[np.lexsort(a.T[::-1])] if len(a) else a


def test_noalloc_matches_allocating_path_twice(geom_full, cuts):
    ctx = lst.Context(0, max_events=2)
    ctx.load_geometry(geom_full, cuts, synth.mlp_flat(synth.xavier_mlp()), 2)
    dev = torch.device("cuda:0")
    events = [synth.pileup_event(geom_full, 7, pileup=120, mean_per_vertex=96),
              synth.pileup_event(geom_full, 8, pileup=200, mean_per_vertex=96)]
    cap = 400_000
    out = torch.full((cap, 2), -1, dtype=torch.int32, device=dev)
    kap = torch.zeros(cap, dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    for e in events:      # two calls in a row, different sizes: the scratch is reused
        t = [torch.from_numpy(a).to(dev) for a in (e.x, e.y, e.z, e.sensor)]
        assert ctx.find_minidoublets_noalloc(*t, out, kap, cnt) == lst.LST_OK
        torch.cuda.synchronize()
        n = int(cnt.item())
        assert 0 < n <= cap
        got = out[:n].cpu().numpy()
        ev = ctx.run_event(*t)
        ref = ev.candidates(lst.LST_MD)
        ev.release()
        assert n == len(ref)
        # integer hit-index work: exact equality of the two sets
        assert np.array_equal(_sorted_rows(got), _sorted_rows(ref))
        # no duplicates
        assert len(np.unique(got, axis=0)) == n
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(geom_full, cuts):
    ctx = lst.Context(0, max_events=1)
    ctx.load_geometry(geom_full, cuts)
    dev = torch.device("cuda:0")
    n = lst.NOALLOC_MAX_HITS + 1
    x = torch.zeros(n, dtype=torch.float32, device=dev)
    s = torch.zeros(n, dtype=torch.int32, device=dev)
    out = torch.zeros((16, 2), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    with pytest.raises(lst.LstError) as ei:
        ctx.find_minidoublets_noalloc(x, x, x, s, out, None, cnt)
    assert ei.value.status == lst.LST_ERR_ARG
    assert "LST_NOALLOC_MAX_HITS" in str(ei.value)
    ctx.close()


def _noalloc_setup(geom_full, cuts, index, pileup):
    ctx = lst.Context(0, max_events=1)
    ctx.load_geometry(geom_full, cuts)
    e = synth.pileup_event(geom_full, index, pileup=pileup, mean_per_vertex=96)
    dev = torch.device("cuda:0")
    t = [torch.from_numpy(a).to(dev) for a in (e.x, e.y, e.z, e.sensor)]
    return ctx, e, t, dev


def test_noalloc_curvatures_equal_the_oracle(geom_full, cuts):
    """The stored MD curvature is the FP32 cut value: bit-equal to the oracle's, pair by pair;
    the call runs on a stream of its own."""
    import oracle
    ctx, e, t, dev = _noalloc_setup(geom_full, cuts, 9, 60)
    cap = 100_000
    out = torch.full((cap, 2), -1, dtype=torch.int32, device=dev)
    kap = torch.full((cap,), float("nan"), dtype=torch.float32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        assert ctx.find_minidoublets_noalloc(*t, out, kap, cnt, stream=stream) == lst.LST_OK
    stream.synchronize()
    n = int(cnt.item())
    ref = oracle.run_event(geom_full, e, cuts)
    assert n == len(ref.md_lo) > 0
    got = out[:n].cpu().numpy()
    gk = kap[:n].cpu().numpy()
    o = np.lexsort(got.T[::-1])
    rh = ref.md_hits()
    ro = np.lexsort(rh.T[::-1])
    assert np.array_equal(got[o], rh[ro])
    assert np.array_equal(gk[o].view(np.uint32), ref.md_kappa[ro].view(np.uint32))
    ctx.close()


def test_noalloc_count_beyond_capacity(geom_full, cuts):
    """With room for half of the MDs the full count is reported and exactly `capacity`
    distinct MDs of the event are written; nothing lands past the buffer's end."""
    ctx, e, t, dev = _noalloc_setup(geom_full, cuts, 10, 40)
    big = torch.full((200_000, 2), -1, dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ctx.find_minidoublets_noalloc(*t, big, None, cnt)
    torch.cuda.synchronize()
    n = int(cnt.item())
    full = {tuple(r) for r in big[:n].cpu().numpy()}
    assert n > 100 and len(full) == n
    cap = n // 2
    guard = torch.full((cap + 64, 2), -7, dtype=torch.int32, device=dev)
    out = guard[:cap]
    assert ctx.find_minidoublets_noalloc(*t, out, None, cnt) == lst.LST_OK
    torch.cuda.synchronize()
    assert int(cnt.item()) == n
    rows = out.cpu().numpy()
    assert len({tuple(r) for r in rows}) == cap and {tuple(r) for r in rows} <= full
    assert (guard[cap:].cpu().numpy() == -7).all()
    ctx.close()


@pytest.mark.parametrize("bad", ["sensor", "nan"])
def test_noalloc_invalid_hit_reports_minus_one(geom_full, cuts, bad):
    """An invalid sensor id or a non-finite coordinate gives md_count = -1 with LST_OK, and
    the next valid call is correct again."""
    ctx, e, t, dev = _noalloc_setup(geom_full, cuts, 11, 20)
    x, y, z, s = [a.clone() for a in t]
    if bad == "sensor":
        s[17] = 2 * geom_full.n_mod
    else:
        x[17] = float("nan")
    out = torch.zeros((100_000, 2), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    assert ctx.find_minidoublets_noalloc(x, y, z, s, out, None, cnt) == lst.LST_OK
    torch.cuda.synchronize()
    assert int(cnt.item()) == -1
    assert ctx.find_minidoublets_noalloc(*t, out, None, cnt) == lst.LST_OK
    torch.cuda.synchronize()
    n = int(cnt.item())
    ev = ctx.run_event(*t)
    ref = ev.candidates(lst.LST_MD)
    ev.release()
    assert n == len(ref) and np.array_equal(_sorted_rows(out[:n].cpu().numpy()), _sorted_rows(ref))
    ctx.close()
