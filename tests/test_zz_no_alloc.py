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
