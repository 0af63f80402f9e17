"""NVTX ranges: with an injection library attached (the mechanism profilers use), the library
names its domain "lst", opens a range for each public call and, inside it, one for each stage
of the launch sequence, and closes every range it opens. The probe (tests/nvtx_probe.c) is
compiled here and the run happens in a child process, which reads NVTX_INJECTION64_PATH at
its first NVTX call."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes as C, sys
sys.path.insert(0, __ROOT__)
import numpy as np
from paper_2403_13166_gb300 import lst, synth
g = synth.build_geometry(False)
ctx = lst.Context(0, max_events=4)
ctx.load_geometry(g, synth.default_cuts())
e = synth.toy_event(g, 1)
ev = ctx.run_event(e.x, e.y, e.z, e.sensor)
ev.candidates(lst.LST_T5)
ev.release()
for h in ctx.run_batch([(e.x, e.y, e.z, e.sensor)] * 2):
    h.counts()
    h.release()
ctx.close()
p = C.CDLL(__PROBE__)
p.nvtx_probe_name.restype = C.c_char_p
p.nvtx_probe_domain.restype = C.c_char_p
n = p.nvtx_probe_pushes()
print("DOMAIN", p.nvtx_probe_domain().decode())
print("COUNTS", n, p.nvtx_probe_pops(), p.nvtx_probe_max_depth())
for i in range(min(n, 4096)):
    print("RANGE", p.nvtx_probe_name(i).decode())
"""


def test_nvtx_ranges_of_calls_and_stages(tmp_path):
    probe = str(tmp_path / "nvtx_probe.so")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-I", cuda_inc, "-o", probe,
                    os.path.join(ROOT, "tests", "nvtx_probe.c")], check=True)
    env = dict(os.environ, NVTX_INJECTION64_PATH=probe)
    code = CHILD.replace("__ROOT__", repr(ROOT)).replace("__PROBE__", repr(probe))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = r.stdout.splitlines()
    domain = [l.split(" ", 1)[1] for l in lines if l.startswith("DOMAIN ")]
    counts = [l.split()[1:] for l in lines if l.startswith("COUNTS ")][0]
    names = [l.split(" ", 1)[1] if " " in l else "" for l in lines if l.startswith("RANGE")]
    pushes, pops, depth = map(int, counts)
    assert domain == ["lst"]
    assert pushes > 0 and pushes == pops and depth >= 2
    for call in ("lst_run_event", "lst_get_candidates", "lst_run_batch"):
        assert call in names, call
    stages = ["hit grouping", "step 1: MD", "step 2: LS", "LS grouping", "step 3: T3", "step 4: T5",
              "T5-DNN score", "track candidates"]
    # the single event's launch sequence: its stage ranges in order, right after its call
    i = names.index("lst_run_event")
    assert names[i + 1:i + 1 + len(stages)] == stages
