"""Build liblst.so (sm_103a) in-tree with nvcc: one object per translation unit, compiled
in parallel, linked as a plain shared library with a C-ABI (see include/lst.h)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblst.so")
SOURCES = ["lst_kernels.cu", "lst_score.cu", "lst_mma.cu", "lst_tc.cu", "lst_pixel.cu", "lst_api.cu",
           "lst_noalloc.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# IEEE FP32 everywhere: no contraction of a*b+c (explicit fmaf only), correctly rounded
# division and square root, denormals kept. The cut arithmetic depends on it.
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
         "-ftz=false", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return False
    t = os.path.getmtime(target)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(verbose: bool = False, force: bool = False, extra_flags=(), out_dir: str = OUT_DIR) -> str:
    """Compile (what is out of date) and link <out_dir>/liblst.so; returns its path. A
    variant build (extra_flags, e.g. -DLST_CHECK for the bounds-checked kernels) must use
    an out_dir of its own."""
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "liblst.so")
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".cuh", ".h"))]
    headers.append(os.path.join(ROOT, "include", "lst.h"))
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not _newer(o, [s] + headers + [__file__]):
            jobs.append([NVCC, *ARCH, *FLAGS, *extra_flags, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if jobs or not _newer(lib, objs):          # also after a link that failed last time
        tmp = lib + f".{os.getpid()}.tmp"
        run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
