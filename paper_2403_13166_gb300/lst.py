"""Thin Python binding of liblst.so (include/lst.h): argument marshalling only.

Every step of the hot path runs in the library's CUDA kernels. Device buffers and streams
come from PyTorch (``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``);
host numpy arrays are accepted where the C-ABI accepts host memory. There is no CPU
fallback: if the library cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblst.so")

LST_OK, LST_ERR_ARG, LST_ERR_CAPACITY, LST_ERR_CUDA, LST_ERR_TIMEOUT, LST_ERR_NOT_READY, \
    LST_ERR_INPUT, LST_ERR_NOMEM = range(8)
LST_MD, LST_LS, LST_T3, LST_T5, LST_TC = range(5)
N_STAGES = 8
GRAPH_NODE_FEATURES, GRAPH_EDGE_FEATURES = 6, 2
STAGES = ("bin", "md", "ls", "ls_group", "t3", "t5", "score", "tc")
LST_FP32, LST_BF16, LST_BF16X3 = 0, 1, 2
WIDTH = {LST_MD: 2, LST_LS: 4, LST_T3: 6, LST_T5: 10, LST_TC: 10}
NFEAT = 38


class LstError(RuntimeError):
    def __init__(self, status, where, msg):
        super().__init__(f"{where}: {_status_str(status)} ({msg})")
        self.status = status


class lst_module(C.Structure):
    _fields_ = [("layer", C.c_int32), ("subdet", C.c_int32), ("side", C.c_int32), ("ps", C.c_int32)]


class lst_cuts(C.Structure):
    _fields_ = [(f, C.c_float) for f in synth.CUT_FIELDS]


class lst_mlp(C.Structure):
    _fields_ = [("n_hidden", C.c_int32), ("w", C.c_void_p)]


class lst_config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_events", C.c_int32), ("use_graphs", C.c_int32),
                ("reserved", C.c_int32), ("md_per_hit", C.c_float), ("ls_per_md", C.c_float),
                ("t3_per_md", C.c_float), ("t5_per_md", C.c_float)]


class lst_launch(C.Structure):
    _fields_ = [(f, C.c_int32) for f in ("md_threads", "md_buf", "ls_threads", "ls_list", "t3_threads",
                                          "t5_threads", "sc_threads", "t3_mds")]


class lst_pixel_cuts(C.Structure):
    _fields_ = [(f, C.c_float) for f in synth.PIXEL_CUT_FIELDS]


class lst_pixel_counts(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("n_pt5", C.c_int64), ("n_t5", C.c_int64), ("n_pt3", C.c_int64),
                ("n_pls", C.c_int64), ("rounds_pt5", C.c_int32), ("rounds_pt3", C.c_int32)]


def pixel_cuts_struct(pc: dict) -> lst_pixel_cuts:
    return lst_pixel_cuts(*[float(np.float32(pc[f])) for f in synth.PIXEL_CUT_FIELDS])


class lst_counts(C.Structure):
    _fields_ = [("n_hits", C.c_int64), ("n_md", C.c_int64), ("n_ls", C.c_int64), ("n_t3", C.c_int64),
                ("n_t5", C.c_int64), ("n_selected", C.c_int64), ("pairs", C.c_int64 * 4),
                ("status", C.c_int32), ("overflow_mask", C.c_int32), ("n_tc", C.c_int64)]


_lib = None
_lock = threading.Lock()

# name -> (restype, argtypes); every function returns lst_status unless stated
_SIGS = {
    "lst_default_config": [C.POINTER(lst_config)],
    "lst_create": [C.c_int, C.POINTER(lst_config), C.POINTER(C.c_void_p)],
    "lst_load_geometry": [C.c_void_p, C.POINTER(lst_module), C.c_int32, C.c_void_p, C.c_void_p,
                          C.POINTER(lst_cuts), C.POINTER(lst_mlp)],
    "lst_run_event": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                      C.POINTER(C.c_void_p)],
    "lst_run_batch": [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                      C.c_void_p, C.c_void_p],
    "lst_event_counts": [C.c_void_p, C.POINTER(lst_counts)],
    "lst_get_candidates": [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                           C.POINTER(C.c_int64)],
    "lst_get_t5_features": [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64)],
    "lst_get_candidates_batch": [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_void_p],
    "lst_get_ls_graph": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64,
                         C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
    "lst_score_t5": [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p],
    "lst_event_release": [C.c_void_p],
    "lst_destroy": [C.c_void_p],
    "lst_set_timing": [C.c_void_p, C.c_int32],
    "lst_set_wait_limit": [C.c_void_p, C.c_int64],
    "lst_device_errors": [C.c_void_p],
    "lst_test_skip_mma": [C.c_void_p, C.c_int32],
    "lst_test_fail_alloc": [C.c_void_p, C.c_int32],
    "lst_match_pixel_seeds": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p],
    "lst_match_pixel_seeds_batch": [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
    "lst_get_pixel_candidates": [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p],
    "lst_get_launch": [C.c_void_p, C.POINTER(lst_launch)],
    "lst_set_launch": [C.c_void_p, C.POINTER(lst_launch)],
    "lst_stage_times": [C.c_void_p, C.c_void_p, C.c_void_p],
    "lst_find_minidoublets_noalloc": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_int64, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                      C.c_void_p],
}

#: limits of lst_find_minidoublets_noalloc's fixed scratch array (include/lst.h)
NOALLOC_MAX_HITS = 524288
NOALLOC_MAX_SENSORS = 32768


def noalloc_arguments(device, x, y, z, sensor, md_hits, md_kappa, md_count):
    """Check the buffers of lst_find_minidoublets_noalloc, whose kernels trust their sizes:
    every buffer a contiguous torch tensor on `device`; x, y, z float32 and sensor int32 of
    one length; md_hits int32 of shape (cap, 2); md_kappa None or float32 with at least cap
    elements; md_count int64 with at least one element. Returns (n_hits, cap); raises
    ValueError naming the first buffer that does not fit."""
    import torch

    def tensor(name, a, dtype):
        if not isinstance(a, torch.Tensor):
            raise ValueError(f"{name}: expected a torch tensor on {device}, got {type(a).__name__}")
        if a.device != device:
            raise ValueError(f"{name}: on {a.device}, expected {device}")
        if a.dtype != dtype:
            raise ValueError(f"{name}: dtype {a.dtype}, expected {dtype}")
        if not a.is_contiguous():
            raise ValueError(f"{name}: not contiguous")
        return a

    n = None
    for name, a, dt in (("x", x, torch.float32), ("y", y, torch.float32), ("z", z, torch.float32),
                        ("sensor", sensor, torch.int32)):
        tensor(name, a, dt)
        if a.dim() != 1:
            raise ValueError(f"{name}: expected one dimension, got shape {tuple(a.shape)}")
        if n is None:
            n = int(a.shape[0])
        elif int(a.shape[0]) != n:
            raise ValueError(f"{name}: length {int(a.shape[0])}, expected {n} (the length of x)")
    tensor("md_hits", md_hits, torch.int32)
    if md_hits.dim() != 2 or int(md_hits.shape[1]) != 2:
        raise ValueError(f"md_hits: expected shape (capacity, 2), got {tuple(md_hits.shape)}")
    cap = int(md_hits.shape[0])
    if md_kappa is not None:
        tensor("md_kappa", md_kappa, torch.float32)
        if md_kappa.numel() < cap:
            raise ValueError(f"md_kappa: {md_kappa.numel()} elements, fewer than the capacity {cap}")
    tensor("md_count", md_count, torch.int64)
    if md_count.numel() < 1:
        raise ValueError("md_count: empty")
    return n, cap


def load_library(path: str = LIB_PATH):
    """Load liblst.so; raises if it is missing (build it with paper_2403_13166_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"liblst.so not built ({path}); run __graft_entry__.build()")
            lib = C.CDLL(path)
            for name, argt in _SIGS.items():
                f = getattr(lib, name)
                f.restype = C.c_int
                f.argtypes = argt
            lib.lst_status_str.restype = C.c_char_p
            lib.lst_status_str.argtypes = [C.c_int32]
            lib.lst_last_error.restype = C.c_char_p
            lib.lst_last_error.argtypes = []
            _lib = lib
    return _lib


def _status_str(s):
    try:
        return load_library().lst_status_str(int(s)).decode()
    except Exception:  # pragma: no cover - only for messages
        return str(s)


def _check(status, where, ok=(LST_OK,)):
    if status not in ok:
        raise LstError(status, where, load_library().lst_last_error().decode())
    return status


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return C.c_void_p(a.ctypes.data)
    raise TypeError(type(a))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except Exception:
            pass
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def default_config(**kw) -> lst_config:
    cfg = lst_config()
    _check(load_library().lst_default_config(C.byref(cfg)), "lst_default_config")
    for k, v in kw.items():
        setattr(cfg, k, v)
    return cfg


def cuts_struct(cuts: dict) -> lst_cuts:
    return lst_cuts(*[float(np.float32(cuts[f])) for f in synth.CUT_FIELDS])


class Event:
    """Handle of one event's results (lst_event)."""

    def __init__(self, ctx, handle, status=LST_OK):
        self.ctx = ctx
        self.h = handle
        self.status = status

    def counts(self) -> dict:
        c = lst_counts()
        _check(load_library().lst_event_counts(self.h, C.byref(c)), "lst_event_counts")
        return dict(n_hits=c.n_hits, md=c.n_md, ls=c.n_ls, t3=c.n_t3, t5=c.n_t5, selected=c.n_selected,
                    tc=c.n_tc, pairs=list(c.pairs), status=c.status, overflow_mask=c.overflow_mask)

    def candidates(self, kind: int, out=None, score=None, selected=None):
        """Hit tuples [n][2|4|6|10] (+ score and selection for T5s and track candidates).
        Host numpy by default; pass torch CUDA tensors to receive device copies."""
        lib = load_library()
        n = C.c_int64(0)
        st = lib.lst_get_candidates(self.h, kind, None, None, None, 0, C.byref(n))
        _check(st, "lst_get_candidates", ok=(LST_OK, LST_ERR_CAPACITY))
        cnt = n.value
        w = WIDTH[kind]
        if out is None:
            out = np.zeros((cnt, w), np.int32)
            if kind in (LST_T5, LST_TC):
                score = np.zeros(cnt, np.float32)
                selected = np.zeros(cnt, np.uint8)
        if cnt:
            _check(lib.lst_get_candidates(self.h, kind, _ptr(out), _ptr(score), _ptr(selected), cnt,
                                          C.byref(n)), "lst_get_candidates")
        if kind in (LST_T5, LST_TC):
            return out, score, selected
        return out

    def match_pixel_seeds(self, seeds, pcuts: dict) -> dict:
        """Table 1 steps 5-8 for this event (lst_match_pixel_seeds): seeds float32 [n][4][3]
        (numpy or a CUDA tensor). Returns the counts per track-candidate type."""
        if hasattr(seeds, "data_ptr"):
            n = int(seeds.shape[0])
            assert seeds.dtype.itemsize == 4 and seeds.is_contiguous() and seeds.numel() == 12 * n
            ptr = _ptr(seeds)
        else:
            seeds = np.ascontiguousarray(seeds, np.float32).reshape(-1, 12)
            n = seeds.shape[0]
            ptr = _ptr(seeds)
        cnt = lst_pixel_counts()
        pc = pixel_cuts_struct(pcuts)
        _check(load_library().lst_match_pixel_seeds(self.h, ptr, n, C.byref(pc), C.byref(cnt)),
               "lst_match_pixel_seeds")
        return {f: getattr(cnt, f) for f, _ in lst_pixel_counts._fields_}

    def pixel_candidates(self) -> np.ndarray:
        """Rows (type 5..8, seed index or -1, T5 / T3 row or -1) of the last matching."""
        lib = load_library()
        n = C.c_int64(0)
        _check(lib.lst_get_pixel_candidates(self.h, None, 0, C.byref(n)), "lst_get_pixel_candidates",
               ok=(LST_OK, LST_ERR_CAPACITY))
        out = np.zeros((n.value, 3), np.int32)
        if n.value:
            _check(lib.lst_get_pixel_candidates(self.h, _ptr(out), n.value, C.byref(n)), "lst_get_pixel_candidates")
        return out

    def features(self):
        lib = load_library()
        n = C.c_int64(0)
        _check(lib.lst_get_t5_features(self.h, None, 0, C.byref(n)), "lst_get_t5_features",
               ok=(LST_OK, LST_ERR_CAPACITY))
        f = np.zeros((n.value, NFEAT), np.float32)
        if n.value:
            _check(lib.lst_get_t5_features(self.h, _ptr(f), n.value, C.byref(n)), "lst_get_t5_features")
        return f

    def ls_graph(self, features=True):
        """The LS graph (MD nodes, LS edges) as host arrays: row_off [n+1], col [m], and with
        features node_feat [n][6] (anchor x, y, z, r, MD curvature, layer) and edge_feat [m][2]
        (LS curvature, chord z at r = 0)."""
        lib = load_library()
        nn, ne = C.c_int64(0), C.c_int64(0)
        _check(lib.lst_get_ls_graph(self.h, None, None, None, None, 0, 0, C.byref(nn), C.byref(ne)),
               "lst_get_ls_graph", ok=(LST_OK, LST_ERR_CAPACITY))
        n, m = nn.value, ne.value
        row = np.zeros(n + 1, np.int32)
        col = np.zeros(max(m, 1), np.int32)
        nf = np.zeros((n, GRAPH_NODE_FEATURES), np.float32) if features else None
        ef = np.zeros((m, GRAPH_EDGE_FEATURES), np.float32) if features else None
        _check(lib.lst_get_ls_graph(self.h, _ptr(row), _ptr(col), _ptr(nf), _ptr(ef), n, m, C.byref(nn),
                                    C.byref(ne)), "lst_get_ls_graph")
        return row, col[:m], nf, ef

    def ls_graph_into(self, row_off, col, node_feat=None, edge_feat=None):
        """Export into caller buffers (torch CUDA tensors or numpy arrays, all of one kind);
        returns (n_nodes, n_edges)."""
        nn, ne = C.c_int64(0), C.c_int64(0)
        _check(load_library().lst_get_ls_graph(self.h, _ptr(row_off), _ptr(col), _ptr(node_feat), _ptr(edge_feat),
                                               int(row_off.shape[0]) - 1, int(col.shape[0]), C.byref(nn),
                                               C.byref(ne)), "lst_get_ls_graph")
        return nn.value, ne.value

    def release(self):
        if self.h:
            load_library().lst_event_release(self.h)
            self.h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


class Context:
    """lst_ctx: device-resident detector, module map, cut parameters and T5-DNN."""

    def __init__(self, device: int = 0, **cfg):
        lib = load_library()
        self._cfg = default_config(**cfg)
        h = C.c_void_p()
        _check(lib.lst_create(device, C.byref(self._cfg), C.byref(h)), "lst_create")
        self.h = h
        self.device = device

    def load_geometry(self, geom, cuts: dict, mlp_flat=None, n_hidden: int = 2):
        lib = load_library()
        n = geom.n_mod
        mods = (lst_module * n)()
        for i in range(n):
            mods[i] = lst_module(int(geom.layer[i]), int(geom.subdet[i]), int(geom.side[i]), int(geom.ps[i]))
        off = np.ascontiguousarray(geom.map_off, np.int32)
        tgt = np.ascontiguousarray(geom.map_tgt, np.int32)
        cs = cuts_struct(cuts)
        mp = None
        self._w = None
        if mlp_flat is not None:
            self._w = np.ascontiguousarray(mlp_flat, np.float32)
            mp = C.byref(lst_mlp(int(n_hidden), self._w.ctypes.data))
        _check(lib.lst_load_geometry(self.h, mods, n, _ptr(off), _ptr(tgt), C.byref(cs), mp),
               "lst_load_geometry")
        self.cuts = dict(cuts)

    def run_event(self, x, y, z, sensor, stream=None) -> Event:
        lib = load_library()
        n = int(x.shape[0])
        ev = C.c_void_p()
        st = lib.lst_run_event(self.h, _ptr(x), _ptr(y), _ptr(z), _ptr(sensor), n, _stream_handle(stream),
                               C.byref(ev))
        _check(st, "lst_run_event", ok=(LST_OK, LST_ERR_INPUT, LST_ERR_TIMEOUT))
        return Event(self, ev, st)

    def run_batch(self, events, stream=None):
        """events: list of (x, y, z, sensor) device tensors or host arrays."""
        lib = load_library()
        n = len(events)
        P = C.c_void_p * n
        xs, ys, zs, ss = P(), P(), P(), P()
        nh = (C.c_int64 * n)()
        for i, (x, y, z, s) in enumerate(events):
            xs[i], ys[i], zs[i], ss[i] = _ptr(x), _ptr(y), _ptr(z), _ptr(s)
            nh[i] = int(x.shape[0])
        out = (C.c_void_p * n)()
        _check(lib.lst_run_batch(self.h, n, xs, ys, zs, ss, nh, _stream_handle(stream), out),
               "lst_run_batch")
        return [Event(self, C.c_void_p(out[i]), LST_ERR_NOT_READY) for i in range(n)]

    def match_pixel_seeds_batch(self, events, seeds, pcuts: dict) -> list:
        """lst_match_pixel_seeds_batch: seeds[i] (float32 [n][4][3], numpy or a CUDA tensor)
        for events[i]; returns the counts per event. Each event's rows are then read with
        its pixel_candidates()."""
        n = len(events)
        keep, ptrs = [], (C.c_void_p * n)()
        ns = (C.c_int64 * n)()
        for i, sd in enumerate(seeds):
            if hasattr(sd, "data_ptr"):
                assert sd.dtype.itemsize == 4 and sd.is_contiguous() and sd.numel() % 12 == 0
                ns[i] = int(sd.numel()) // 12
            else:
                sd = np.ascontiguousarray(sd, np.float32).reshape(-1, 12)
                ns[i] = sd.shape[0]
            keep.append(sd)
            ptrs[i] = _ptr(sd) if ns[i] else None
        evs = (C.c_void_p * n)(*[e.h for e in events])
        cnt = (lst_pixel_counts * n)()
        pc = pixel_cuts_struct(pcuts)
        _check(load_library().lst_match_pixel_seeds_batch(evs, n, ptrs, ns, C.byref(pc), cnt),
               "lst_match_pixel_seeds_batch")
        return [{f: getattr(c, f) for f, _ in lst_pixel_counts._fields_} for c in cnt]

    def candidates_batch(self, events, kind: int, out=None, score=None, selected=None):
        """Objects of several events in one call (lst_get_candidates_batch): returns (hits,
        score, selected, offsets) with rows offsets[i]:offsets[i+1] for events[i]. Pass
        preallocated (e.g. pinned) numpy buffers or torch CUDA tensors to avoid allocation;
        they must hold all rows."""
        lib = load_library()
        n = len(events)
        handles = (C.c_void_p * n)(*[e.h for e in events])
        offs = np.zeros(n + 1, np.int64)
        st = lib.lst_get_candidates_batch(handles, n, kind, None, None, None, 0, _ptr(offs))
        _check(st, "lst_get_candidates_batch", ok=(LST_OK, LST_ERR_CAPACITY))
        total = int(offs[-1])
        t5like = kind in (LST_T5, LST_TC)
        if out is None:
            out = np.zeros((total, WIDTH[kind]), np.int32)
            if t5like:
                score = np.zeros(total, np.float32)
                selected = np.zeros(total, np.uint8)
        cap = int(out.shape[0])
        if total:
            _check(lib.lst_get_candidates_batch(handles, n, kind, _ptr(out), _ptr(score), _ptr(selected), cap,
                                                _ptr(offs)), "lst_get_candidates_batch")
        return out, score, selected, offs

    def score_t5(self, feat, out, precision=LST_FP32, stream=None):
        lib = load_library()
        _check(lib.lst_score_t5(self.h, _ptr(feat), int(feat.shape[0]), precision, _ptr(out),
                                _stream_handle(stream)), "lst_score_t5")

    def find_minidoublets_noalloc(self, x, y, z, sensor, md_hits, md_kappa, md_count, stream=None) -> int:
        """Steps 0-1 without any device allocation by the library (for callers that cannot
        allocate while they run, e.g. inside a framework that owns all device memory). All
        buffers are the caller's device tensors: md_hits int32 [cap, 2], md_kappa float32
        [cap] or None, md_count int64 [1] (count found, or -1 for an invalid hit).
        Returns the lst_status; raises ValueError for a buffer of the wrong kind, type,
        shape or device (before anything is launched) and LstError on other failures."""
        import torch
        n, cap = noalloc_arguments(torch.device("cuda", self.device), x, y, z, sensor, md_hits, md_kappa,
                                   md_count)
        st = load_library().lst_find_minidoublets_noalloc(
            self.h, _ptr(x), _ptr(y), _ptr(z), _ptr(sensor), n, _ptr(md_hits), _ptr(md_kappa),
            cap, _ptr(md_count), _stream_handle(stream))
        return _check(st, "lst_find_minidoublets_noalloc")

    def get_launch(self) -> dict:
        p = lst_launch()
        _check(load_library().lst_get_launch(self.h, C.byref(p)), "lst_get_launch")
        return {f: getattr(p, f) for f, _ in lst_launch._fields_}

    def set_launch(self, **kw):
        cur = self.get_launch()
        cur.update(kw)
        p = lst_launch(**cur)
        _check(load_library().lst_set_launch(self.h, C.byref(p)), "lst_set_launch")

    def set_wait_limit(self, iterations: int):
        _check(load_library().lst_set_wait_limit(self.h, int(iterations)), "lst_set_wait_limit")

    def test_skip_mma(self, on=True):
        """Failure-handling test aid: the tensor-core score kernels issue no MMA, so their
        bounded waits run out (LST_ERR_TIMEOUT) with nothing in flight."""
        _check(load_library().lst_test_skip_mma(self.h, int(on)), "lst_test_skip_mma")

    def test_fail_alloc(self, n=1):
        """Failure-handling test aid: the next n event-buffer allocations fail as if the
        device were out of memory (LST_ERR_NOMEM); n = 0 clears them."""
        _check(load_library().lst_test_fail_alloc(self.h, int(n)), "lst_test_fail_alloc")

    def device_errors(self) -> int:
        return load_library().lst_device_errors(self.h)

    def set_timing(self, on=True):
        _check(load_library().lst_set_timing(self.h, int(on)), "lst_set_timing")

    def stage_times(self):
        """Mean device ms per launch of each of STAGES, and the launch count."""
        a = np.zeros(N_STAGES, np.float32)
        n = C.c_int64(0)
        _check(load_library().lst_stage_times(self.h, _ptr(a), C.byref(n)), "lst_stage_times")
        return a, n.value

    def close(self):
        if getattr(self, "h", None):
            load_library().lst_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# C-ABI names, for callers that prefer the flat interface
def lst_create(device=0, **cfg):
    return Context(device, **cfg)


def lst_load_geometry(ctx, geom, cuts, mlp_flat=None, n_hidden=2):
    ctx.load_geometry(geom, cuts, mlp_flat, n_hidden)


def lst_run_event(ctx, x, y, z, sensor, stream=None):
    return ctx.run_event(x, y, z, sensor, stream)


def lst_run_batch(ctx, events, stream=None):
    return ctx.run_batch(events, stream)


def lst_get_candidates(ev, kind):
    return ev.candidates(kind)


def lst_get_t5_features(ev):
    return ev.features()


def lst_score_t5(ctx, feat, out, precision=LST_FP32, stream=None):
    ctx.score_t5(feat, out, precision, stream)


def lst_event_release(ev):
    ev.release()


def lst_destroy(ctx):
    ctx.close()


def header_symbols(header_path: str):
    """Entry points declared in include/lst.h."""
    import re
    src = open(header_path).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(lst_\w+)\s*\(", src, re.M)))


# ------------------------------------------------------------------ serving
class lst_serve_config(C.Structure):
    _fields_ = [("max_batch", C.c_int32), ("lanes", C.c_int32), ("mem_budget_bytes", C.c_int64),
                ("copy_t5", C.c_int32), ("slot_hits", C.c_int32)]


class lst_serve_result(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("reserved", C.c_int32), ("counts", lst_counts),
                ("t_arrival", C.c_double), ("t_admit", C.c_double), ("t_launch", C.c_double),
                ("t_done", C.c_double), ("n_t5", C.c_int64), ("t5_hits", C.c_void_p),
                ("t5_score", C.c_void_p), ("t5_sel", C.c_void_p), ("owner", C.c_void_p)]


def _serve_sigs(lib):
    lib.lst_clock.restype = C.c_double
    lib.lst_clock.argtypes = []
    for name, argt in {
        "lst_serve_start": [C.c_void_p, C.POINTER(lst_serve_config), C.POINTER(C.c_void_p)],
        "lst_serve_submit": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                             C.c_uint64, C.c_double],
        "lst_serve_poll": [C.c_void_p, C.POINTER(lst_serve_result), C.c_int32, C.POINTER(C.c_int32), C.c_int32],
        "lst_serve_free_result": [C.POINTER(lst_serve_result)],
        "lst_serve_stop": [C.c_void_p],
    }.items():
        f = getattr(lib, name)
        f.restype = C.c_int
        f.argtypes = argt
    return lib


def clock() -> float:
    """lst_clock(): the library's monotonic clock in seconds."""
    return _serve_sigs(load_library()).lst_clock()


class Server:
    """lst_serve_*: continuous batching of events submitted one at a time (host arrays)."""

    def __init__(self, ctx: Context, max_batch=32, lanes=2, mem_budget_bytes=8 << 30, copy_t5=True, slot_hits=0):
        lib = _serve_sigs(load_library())
        cfg = lst_serve_config(int(max_batch), int(lanes), int(mem_budget_bytes), int(bool(copy_t5)), int(slot_hits))
        h = C.c_void_p()
        _check(lib.lst_serve_start(ctx.h, C.byref(cfg), C.byref(h)), "lst_serve_start")
        self.h = h
        self.ctx = ctx
        self._keep = {}
        self._buf = (lst_serve_result * 256)()

    def submit(self, x, y, z, sensor, tag: int, t_arrival: float = 0.0):
        arrs = [np.ascontiguousarray(a) for a in (x, y, z, sensor)]
        self._keep[int(tag)] = arrs
        _check(load_library().lst_serve_submit(self.h, *[_ptr(a) for a in arrs], int(arrs[0].shape[0]), int(tag),
                                               float(t_arrival)), "lst_serve_submit")

    def poll(self, wait_ms: int = 0, max_results: int = 256, keep_t5: bool = True):
        """Finished requests as dicts. With keep_t5 the T5 tuples, scores and selection flags
        are copied out of the library's pinned staging into numpy arrays; without, only the
        counts and times are kept. Either way the staging is released before returning."""
        lib = load_library()
        n = C.c_int32(0)
        _check(lib.lst_serve_poll(self.h, self._buf, min(max_results, 256), C.byref(n), int(wait_ms)),
               "lst_serve_poll")
        out = []
        for i in range(n.value):
            r = self._buf[i]
            d = dict(tag=r.tag, status=r.status, t_arrival=r.t_arrival, t_admit=r.t_admit, t_launch=r.t_launch,
                     t_done=r.t_done, n_t5=r.n_t5, t5=r.counts.n_t5, md=r.counts.n_md, ls=r.counts.n_ls,
                     t3=r.counts.n_t3, selected=r.counts.n_selected, tc=r.counts.n_tc)
            if keep_t5 and r.t5_hits and r.n_t5:
                n5 = r.n_t5
                d["t5_hits"] = np.ctypeslib.as_array((C.c_int32 * (n5 * 10)).from_address(r.t5_hits)).reshape(n5, 10).copy()
                d["t5_score"] = np.ctypeslib.as_array((C.c_float * n5).from_address(r.t5_score)).copy()
                d["t5_sel"] = np.ctypeslib.as_array((C.c_uint8 * n5).from_address(r.t5_sel)).copy()
            lib.lst_serve_free_result(C.byref(r))
            self._keep.pop(int(r.tag), None)
            out.append(d)
        return out

    def stop(self):
        if getattr(self, "h", None):
            load_library().lst_serve_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass
