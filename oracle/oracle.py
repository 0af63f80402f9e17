"""ctypes front end of the C oracle (test infrastructure only; see package docstring)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lst_oracle.c")
_LIB = os.path.join(_HERE, "liblst_oracle.so")
_lock = threading.Lock()
_lib = None

CUT_FIELDS = ("kappa_max", "z_lum", "hit_err", "sensor_gap", "t3_kappa_factor", "t3_rz_tol",
              "t5_kappa_rel", "t5_kappa_abs", "t5_rz_tol", "t5_chi2_max", "hit_sigma",
              "k_field", "wp")
NFEAT = 38
NHID = 32


class _Cuts(C.Structure):
    _fields_ = [(f, C.c_float) for f in CUT_FIELDS]


class _Geom(C.Structure):
    _fields_ = [("n_mod", C.c_int32), ("layer", C.c_void_p), ("subdet", C.c_void_p),
                ("side", C.c_void_p), ("map_off", C.c_void_p), ("map_tgt", C.c_void_p)]


class _Mlp(C.Structure):
    _fields_ = [("n_hidden", C.c_int32), ("w", C.c_void_p)]


class _Result(C.Structure):
    _fields_ = [("n_md", C.c_int64), ("n_ls", C.c_int64), ("n_t3", C.c_int64), ("n_t5", C.c_int64),
                ("pairs", C.c_int64 * 4), ("near", C.c_int64 * 4),
                ("md_lo", C.c_void_p), ("md_up", C.c_void_p), ("md_mod", C.c_void_p),
                ("md_kappa", C.c_void_p),
                ("ls_in", C.c_void_p), ("ls_out", C.c_void_p), ("ls_kappa", C.c_void_p),
                ("t3_ls1", C.c_void_p), ("t3_ls2", C.c_void_p), ("t3_md", C.c_void_p),
                ("t3_kappa", C.c_void_p),
                ("t5_t3a", C.c_void_p), ("t5_t3b", C.c_void_p), ("t5_md", C.c_void_p),
                ("t5_feat", C.c_void_p), ("t5_score", C.c_void_p), ("t5_sel", C.c_void_p),
                ("t5_chi2", C.c_void_p), ("t5_tc", C.c_void_p),
                ("n_pix", C.c_int64), ("pix_tc", C.c_void_p), ("pix_ties", C.c_int64)]


PIXEL_CUT_FIELDS = ("kappa_rel", "kappa_abs", "rz_tol", "dphi0", "dphi_cm", "dm_abs", "dm_rel")


class _PCuts(C.Structure):
    _fields_ = [(f, C.c_float) for f in PIXEL_CUT_FIELDS]


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc: no fast-math, no floating-point contraction."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-fexcess-precision=standard", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build_oracle())
            lib.oracle_run.restype = C.c_int
            lib.oracle_run.argtypes = [C.POINTER(_Geom), C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int64, C.POINTER(_Cuts), C.POINTER(_Mlp),
                                       C.c_int, C.c_void_p, C.c_int64, C.POINTER(_PCuts),
                                       C.POINTER(_Result)]
            lib.oracle_pixel_match.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                               C.POINTER(_PCuts), C.c_void_p]
            lib.oracle_free.argtypes = [C.POINTER(_Result)]
            lib.oracle_md_cut.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(_Cuts),
                                          C.POINTER(C.c_float)]
            lib.oracle_ls_cut.argtypes = [C.c_void_p, C.c_void_p, C.c_float, C.c_float, C.c_int,
                                          C.c_int, C.POINTER(_Cuts), C.POINTER(C.c_float)]
            lib.oracle_t3_cut.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(_Cuts),
                                          C.POINTER(C.c_float)]
            lib.oracle_t5_cut.argtypes = [C.c_void_p, C.c_float, C.c_float, C.POINTER(_Cuts)]
            lib.oracle_tc_select.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_int64, C.c_int, C.c_void_p]
            lib.oracle_t5_chi2.restype = C.c_float
            lib.oracle_t5_chi2.argtypes = [C.c_void_p, C.c_float]
            lib.oracle_t5_features.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                               C.c_void_p]
            lib.oracle_mlp.restype = C.c_double
            lib.oracle_mlp.argtypes = [C.POINTER(_Mlp), C.c_void_p]
            _lib = lib
    return _lib


def _cuts(cuts: dict) -> _Cuts:
    return _Cuts(*[float(np.float32(cuts[f])) for f in CUT_FIELDS])


def _f32(a, n):
    a = np.ascontiguousarray(a, np.float32)
    assert a.shape == (n,)
    return a


def md_cut(L, U, endcap, cuts):
    """One mini-doublet test; L, U = (x, y, z, r) float32. Returns (passed, kappa)."""
    lib = _load()
    L, U = _f32(L, 4), _f32(U, 4)
    k = C.c_float(0.0)
    ok = lib.oracle_md_cut(L.ctypes.data, U.ctypes.data, int(endcap), C.byref(_cuts(cuts)), C.byref(k))
    return bool(ok), np.float32(k.value)


def ls_cut(A, B, kA, kB, bA, bB, cuts):
    lib = _load()
    A, B = _f32(A, 4), _f32(B, 4)
    k = C.c_float(0.0)
    ok = lib.oracle_ls_cut(A.ctypes.data, B.ctypes.data, float(kA), float(kB), int(bA), int(bB),
                           C.byref(_cuts(cuts)), C.byref(k))
    return bool(ok), np.float32(k.value)


def t3_cut(P0, P1, P2, cuts):
    lib = _load()
    P0, P1, P2 = _f32(P0, 4), _f32(P1, 4), _f32(P2, 4)
    k = C.c_float(0.0)
    ok = lib.oracle_t3_cut(P0.ctypes.data, P1.ctypes.data, P2.ctypes.data, C.byref(_cuts(cuts)),
                           C.byref(k))
    return bool(ok), np.float32(k.value)


def t5_cut(P, ka, kb, cuts):
    lib = _load()
    P = _f32(np.asarray(P).ravel(), 20)
    return bool(lib.oracle_t5_cut(P.ctypes.data, float(ka), float(kb), C.byref(_cuts(cuts))))


def _pcuts(pcuts: dict) -> _PCuts:
    return _PCuts(*[float(np.float32(pcuts[f])) for f in PIXEL_CUT_FIELDS])


def pixel_match(H, P0, P1, ko, pcuts):
    """One seed / object match: H the seed's hits [4][3], P0 and P1 the object's first two
    anchors (x, y, z, r), ko its curvature (float32). Returns (matched, rz residual,
    |kx - ko|)."""
    lib = _load()
    H = _f32(np.asarray(H).ravel(), 12)
    P0, P1 = _f32(P0, 4), _f32(P1, 4)
    r = (C.c_float * 2)()
    ok = lib.oracle_pixel_match(H.ctypes.data, P0.ctypes.data, P1.ctypes.data, float(np.float32(ko)),
                                C.byref(_pcuts(pcuts)), r)
    return bool(ok), np.float32(r[0]), np.float32(r[1])


def t5_chi2(P, sigma):
    """Circle-fit chi2 of five anchors P[5][4] = (x, y, z, r) float32 (pre-DNN selection)."""
    lib = _load()
    P = _f32(np.asarray(P).ravel(), 20)
    return np.float32(lib.oracle_t5_chi2(P.ctypes.data, float(np.float32(sigma))))


def tc_select(md, key, q, sel, n_md, brute=False):
    """Track-candidate flags of T5s given their MD ids [n][5], hit keys [n][10], circle-fit
    chi2 [n] (float32) and selection flags [n] (duplicate removal by shared MDs)."""
    lib = _load()
    md = np.ascontiguousarray(md, np.int32).reshape(-1, 5)
    n = md.shape[0]
    key = np.ascontiguousarray(key, np.int32).reshape(n, 10)
    q = np.ascontiguousarray(q, np.float32).reshape(n)
    sel = np.ascontiguousarray(sel, np.uint8).reshape(n)
    tc = np.zeros(max(n, 1), np.uint8)
    lib.oracle_tc_select(n, md.ctypes.data, key.ctypes.data, q.ctypes.data, sel.ctypes.data, int(n_md),
                         int(brute), tc.ctypes.data)
    return tc[:n]


def t5_features(anchors, layers, md_kappa, k_field):
    lib = _load()
    a = np.ascontiguousarray(np.asarray(anchors, np.float64).reshape(15))
    lay = np.ascontiguousarray(np.asarray(layers, np.int32).reshape(5))
    mk = np.ascontiguousarray(np.asarray(md_kappa, np.float64).reshape(5))
    f = np.zeros(NFEAT, np.float64)
    lib.oracle_t5_features(a.ctypes.data, lay.ctypes.data, mk.ctypes.data, float(k_field),
                           f.ctypes.data)
    return f


def _mlp_struct(flat: np.ndarray, n_hidden: int):
    w = np.ascontiguousarray(flat, np.float64)
    expect = NHID * NFEAT + NHID + (n_hidden - 1) * (NHID * NHID + NHID) + NHID + 1
    assert w.shape == (expect,), (w.shape, expect)
    return _Mlp(int(n_hidden), w.ctypes.data), w


def mlp_forward(flat: np.ndarray, n_hidden: int, feat: np.ndarray) -> float:
    lib = _load()
    m, keep = _mlp_struct(flat, n_hidden)
    f = np.ascontiguousarray(feat, np.float64).reshape(NFEAT)
    return float(lib.oracle_mlp(C.byref(m), f.ctypes.data))


@dataclass
class OracleResult:
    pairs: np.ndarray
    near: np.ndarray        # tested pairs per step with a tolerance comparison within 1e-5 of its bound
    md_lo: np.ndarray
    md_up: np.ndarray
    md_mod: np.ndarray
    md_kappa: np.ndarray
    ls_in: np.ndarray
    ls_out: np.ndarray
    ls_kappa: np.ndarray
    t3_md: np.ndarray
    t3_kappa: np.ndarray
    t5_md: np.ndarray
    t5_t3a: np.ndarray
    t5_t3b: np.ndarray
    t5_feat: np.ndarray
    t5_score: np.ndarray
    t5_sel: np.ndarray
    t5_chi2: np.ndarray
    t5_tc: np.ndarray
    pix_tc: np.ndarray = None      # [n][3] (type 5/6/7/8, pLS index or -1, T5 / T3 index or -1)
    pix_ties: int = 0

    @property
    def counts(self):
        return dict(md=len(self.md_lo), ls=len(self.ls_in), t3=len(self.t3_kappa), t5=len(self.t5_score))

    # canonical hit tuples (original hit indices), the unit of comparison between implementations
    def md_hits(self):
        return np.stack([self.md_lo, self.md_up], 1)

    def ls_hits(self):
        return np.concatenate([self.md_hits()[self.ls_in], self.md_hits()[self.ls_out]], 1)

    def t3_hits(self):
        mh = self.md_hits()
        return np.concatenate([mh[self.t3_md[:, i]] for i in range(3)], 1)

    def t5_hits(self):
        mh = self.md_hits()
        if len(self.t5_md) == 0:
            return np.zeros((0, 10), np.int32)
        return np.concatenate([mh[self.t5_md[:, i]] for i in range(5)], 1)

    def tc_hits(self):
        return self.t5_hits()[self.t5_tc.astype(bool)]

    def pixel_tcs(self):
        """Steps 5-8 as comparable tuples: (type, pLS index, the object's hit indices padded
        with -1 to 10)."""
        out = []
        if self.pix_tc is None:
            return out
        t5h, t3h = self.t5_hits(), self.t3_hits()
        for typ, p, o in self.pix_tc.tolist():
            h = t5h[o].tolist() if typ in (5, 6) else t3h[o].tolist() if typ == 7 else []
            out.append((typ, p, *(h + [-1] * (10 - len(h)))))
        return out


def _arr(ptr, n, dtype, shape=None):
    if n == 0:
        return np.zeros((0,) + (shape or ()), dtype)
    count = n * (int(np.prod(shape)) if shape else 1)
    buf = (C.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr)
    a = np.frombuffer(buf, dtype=dtype, count=count).copy()
    return a.reshape((n,) + shape) if shape else a


def run_event(geom, event, cuts: dict, mlp_flat=None, n_hidden=2, brute=False, pls=None,
              pcuts=None) -> OracleResult:
    """Run steps 1-4 and the score on one event (all arrays copied out); with pixel seeds
    (pls: float32 [n][4][3]) and their matching parameters also the track candidates of
    steps 5-8."""
    lib = _load()
    layer = np.ascontiguousarray(geom.layer, np.int32)
    subdet = np.ascontiguousarray(geom.subdet, np.int32)
    side = np.ascontiguousarray(geom.side, np.int32)
    moff = np.ascontiguousarray(geom.map_off, np.int32)
    mtgt = np.ascontiguousarray(geom.map_tgt, np.int32)
    g = _Geom(geom.n_mod, layer.ctypes.data, subdet.ctypes.data, side.ctypes.data,
              moff.ctypes.data, mtgt.ctypes.data)
    x = np.ascontiguousarray(event.x, np.float32)
    y = np.ascontiguousarray(event.y, np.float32)
    z = np.ascontiguousarray(event.z, np.float32)
    s = np.ascontiguousarray(event.sensor, np.int32)
    keep = None
    mp = None
    if mlp_flat is not None:
        m, keep = _mlp_struct(mlp_flat, n_hidden)
        mp = C.byref(m)
    res = _Result()
    pk, npl, pcp = None, 0, None
    if pls is not None:
        pk = np.ascontiguousarray(pls, np.float32).reshape(-1, 12)
        npl = pk.shape[0]
        pcp = C.byref(_pcuts(pcuts))
    rc = lib.oracle_run(C.byref(g), x.ctypes.data, y.ctypes.data, z.ctypes.data, s.ctypes.data,
                        x.shape[0], C.byref(_cuts(cuts)), mp, int(brute),
                        pk.ctypes.data if pk is not None else None, npl, pcp, C.byref(res))
    if rc != 0:
        raise ValueError("oracle: invalid hit (sensor id out of range or non-finite coordinate)")
    try:
        n1, n2, n3, n4 = res.n_md, res.n_ls, res.n_t3, res.n_t5
        out = OracleResult(
            pairs=np.array(list(res.pairs), np.int64), near=np.array(list(res.near), np.int64),
            md_lo=_arr(res.md_lo, n1, np.int32), md_up=_arr(res.md_up, n1, np.int32),
            md_mod=_arr(res.md_mod, n1, np.int32), md_kappa=_arr(res.md_kappa, n1, np.float32),
            ls_in=_arr(res.ls_in, n2, np.int32), ls_out=_arr(res.ls_out, n2, np.int32),
            ls_kappa=_arr(res.ls_kappa, n2, np.float32),
            t3_md=_arr(res.t3_md, n3, np.int32, (3,)), t3_kappa=_arr(res.t3_kappa, n3, np.float32),
            t5_md=_arr(res.t5_md, n4, np.int32, (5,)), t5_t3a=_arr(res.t5_t3a, n4, np.int32),
            t5_t3b=_arr(res.t5_t3b, n4, np.int32),
            t5_feat=_arr(res.t5_feat, n4, np.float64, (NFEAT,)),
            t5_score=_arr(res.t5_score, n4, np.float64), t5_sel=_arr(res.t5_sel, n4, np.uint8),
            t5_chi2=_arr(res.t5_chi2, n4, np.float32), t5_tc=_arr(res.t5_tc, n4, np.uint8),
            pix_tc=_arr(res.pix_tc, res.n_pix, np.int32, (3,)) if pls is not None else None,
            pix_ties=int(res.pix_ties))
    finally:
        lib.oracle_free(C.byref(res))
    del keep
    return out
