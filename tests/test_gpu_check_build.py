"""The bounds-checked build (-DLST_CHECK): every data-derived index in the kernels is checked
against its buffer's capacity and a failure is recorded instead of used. The build must
produce exactly the oracle's candidate sets with no check failing, on the toy event and on
a pile-up slice, through the single-event and the batched (graph) paths. It runs in a
process of its own because a process loads one copy of the library."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
sys.path.insert(0, __ROOT__)
import numpy as np
import torch
import oracle
from paper_2403_13166_gb300 import build, lst, synth

path = build.build(extra_flags=["-DLST_CHECK"], out_dir=__OUT__)
lst.load_library(path)
assert lst.load_library()._name == path

def canon(a):
    return a[np.lexsort(a.T[::-1])] if len(a) else a

def same(ev, ref):
    c = ev.counts()
    assert c["status"] == lst.LST_OK, c
    for kind, name in ((lst.LST_MD, "md_hits"), (lst.LST_LS, "ls_hits"), (lst.LST_T3, "t3_hits"),
                       (lst.LST_T5, "t5_hits")):
        got = ev.candidates(kind)
        got = got[0] if isinstance(got, tuple) else got
        assert np.array_equal(canon(got), canon(getattr(ref, name)())), name

w = synth.mlp_flat(synth.xavier_mlp())
cuts = synth.default_cuts()
n = 0
for full, events in ((False, lambda g: [synth.toy_event(g, 0)]),
                     (True, lambda g: [synth.pileup_event(g, 21, pileup=20, mean_per_vertex=96),
                                       synth.pileup_event(g, 22, pileup=5, mean_per_vertex=96)])):
    g = synth.build_geometry(full)
    ctx = lst.Context(0, max_events=4)
    ctx.load_geometry(g, cuts, w, 2)
    evs = events(g)
    refs = [oracle.run_event(g, e, cuts, w, 2) for e in evs]
    dev = [[torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (e.x, e.y, e.z, e.sensor)] for e in evs]
    for d, ref in zip(dev, refs):
        ev = ctx.run_event(*d)
        same(ev, ref)
        ev.release()
        n += 1
    hs = ctx.run_batch(dev)
    for h, ref in zip(hs, refs):
        same(h, ref)
        h.release()
        n += 1
    assert ctx.device_errors() == lst.LST_OK
    ctx.close()
print("CHECKED", n)
"""


def test_bounds_checked_build_matches_the_oracle():
    out = os.path.join(ROOT, "paper_2403_13166_gb300", "_lib_check")
    code = SCRIPT.replace("__ROOT__", repr(ROOT)).replace("__OUT__", repr(out))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "CHECKED 6" in r.stdout
