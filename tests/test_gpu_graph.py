"""GPU: the LS graph export (Section 4: MDs as nodes, LSs as edges) against the oracle's
MDs and LSs: edge set identical, node and edge features identical (FP32 values of the
same expressions), host and device outputs identical, empty events and capacity errors."""
import numpy as np
import pytest

import oracle
from paper_2403_13166_gb300 import lst, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def canon(a):
    return a[np.lexsort(a.T[::-1])] if len(a) else a


@pytest.fixture(scope="module")
def ctx(geom_full, cuts):
    c = lst.Context(0, max_events=4)
    c.load_geometry(geom_full, cuts, synth.mlp_flat(synth.xavier_mlp()), 2)
    yield c
    c.close()


def test_ls_graph_matches_the_oracle(ctx, geom_full, cuts):
    e = synth.pileup_event(geom_full, 7, pileup=80, mean_per_vertex=96)
    ref = oracle.run_event(geom_full, e, cuts, None)
    ev = ctx.run_event(e.x, e.y, e.z, e.sensor)
    md = ev.candidates(lst.LST_MD)
    row, col, nf, ef = ev.ls_graph()
    n, m = len(md), len(col)
    assert n == ref.counts["md"] and m == ref.counts["ls"] and row[0] == 0 and row[-1] == m
    assert np.all(np.diff(row) >= 0)
    src = np.repeat(np.arange(n), np.diff(row))
    edges = np.concatenate([md[src], md[col]], 1)
    assert np.array_equal(canon(edges), canon(ref.ls_hits()))
    # node features: anchor hit, r, curvature (the FP32 cut value), layer
    lo = md[:, 0]
    x, y, z = e.x[lo], e.y[lo], e.z[lo]
    r = np.sqrt(x * x + y * y)
    assert np.array_equal(nf[:, :4], np.stack([x, y, z, r], 1))
    oidx = {(a, b): i for i, (a, b) in enumerate(ref.md_hits())}
    perm = np.array([oidx[(a, b)] for a, b in md])
    assert np.array_equal(nf[:, 4], ref.md_kappa[perm])
    assert np.array_equal(nf[:, 5], geom_full.layer[ref.md_mod[perm]].astype(np.float32))
    # edge features: LS curvature and the chord's z at r = 0 (FP32 expression)
    lidx = {tuple(h): i for i, h in enumerate(ref.ls_hits())}
    lperm = np.array([lidx[tuple(h)] for h in edges])
    assert np.array_equal(ef[:, 0], ref.ls_kappa[lperm])
    za, ra, zb, rb = nf[src, 2], nf[src, 3], nf[col, 2], nf[col, 3]
    with np.errstate(all="ignore"):
        z0 = za - ra * ((zb - za) / (rb - ra))
    assert np.array_equal(ef[:, 1], z0.astype(np.float32))
    ev.release()


def test_device_buffers_and_edge_cases(ctx, geom_full):
    e = synth.pileup_event(geom_full, 8, pileup=20, mean_per_vertex=96)
    ev = ctx.run_event(e.x, e.y, e.z, e.sensor)
    row, col, nf, ef = ev.ls_graph()
    n, m = len(row) - 1, len(col)
    d = [torch.zeros(n + 1, dtype=torch.int32, device="cuda"), torch.zeros(m, dtype=torch.int32, device="cuda"),
         torch.zeros((n, 6), dtype=torch.float32, device="cuda"), torch.zeros((m, 2), dtype=torch.float32, device="cuda")]
    lib = lst.load_library()
    import ctypes as C
    nn, ne = C.c_int64(0), C.c_int64(0)
    st = lib.lst_get_ls_graph(ev.h, *[C.c_void_p(t.data_ptr()) for t in d], n, m, C.byref(nn), C.byref(ne))
    assert st == lst.LST_OK and nn.value == n and ne.value == m
    torch.cuda.synchronize()
    assert np.array_equal(d[0].cpu().numpy(), row)
    # edges of one node come in no particular order: compare per-row sorted
    dc = d[1].cpu().numpy()
    for i in range(0, n, max(1, n // 500)):
        assert np.array_equal(np.sort(dc[row[i]:row[i + 1]]), np.sort(col[row[i]:row[i + 1]]))
    assert np.array_equal(d[2].cpu().numpy(), nf)
    # too small: nothing copied, counts reported
    st = lib.lst_get_ls_graph(ev.h, *[C.c_void_p(t.data_ptr()) for t in d], n - 1, m, C.byref(nn), C.byref(ne))
    assert st == lst.LST_ERR_CAPACITY and nn.value == n
    ev.release()
    empty = ctx.run_event(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32),
                          np.zeros(0, np.int32))
    row, col, nf, ef = empty.ls_graph()
    assert list(row) == [0] and len(col) == 0
    empty.release()
