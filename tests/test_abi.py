"""The C-ABI library builds, loads and exports every entry point declared in include/lst.h
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2403_13166_gb300 import build
    return build.build()


def test_header_symbols_exported(libpath):
    from paper_2403_13166_gb300 import lst
    syms = lst.header_symbols(os.path.join(ROOT, "include", "lst.h"))
    for must in ("lst_load_geometry", "lst_run_event", "lst_get_candidates", "lst_score_t5",
                 "lst_create", "lst_destroy", "lst_run_batch"):
        assert must in syms
    lib = ctypes.CDLL(libpath)
    for s in syms:
        assert hasattr(lib, s), s
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(syms) <= exported


def test_binding_loads_and_reports_status(libpath):
    from paper_2403_13166_gb300 import lst
    lib = lst.load_library()
    assert lib.lst_status_str(lst.LST_ERR_CAPACITY).decode() == "LST_ERR_CAPACITY"
    assert lib.lst_status_str(99).decode() == "LST_ERR_UNKNOWN"
    cfg = lst.default_config()
    assert cfg.max_events >= 1 and cfg.precision == lst.LST_FP32
    # argument checks need no device
    h = ctypes.c_void_p()
    assert lib.lst_create(0, None, None) == lst.LST_ERR_ARG
    assert lib.lst_run_event(None, None, None, None, None, 0, None, ctypes.byref(h)) == lst.LST_ERR_ARG


def test_binding_names_match_abi(libpath):
    from paper_2403_13166_gb300 import lst
    for name in ("lst_create", "lst_load_geometry", "lst_run_event", "lst_run_batch", "lst_get_candidates",
                 "lst_get_t5_features", "lst_score_t5", "lst_event_release", "lst_destroy"):
        assert callable(getattr(lst, name))


def test_structs_match_header_layout(libpath):
    from paper_2403_13166_gb300 import lst
    assert ctypes.sizeof(lst.lst_cuts) == 13 * 4
    assert ctypes.sizeof(lst.lst_module) == 16
    assert ctypes.sizeof(lst.lst_config) == 32
    assert ctypes.sizeof(lst.lst_counts) == 10 * 8 + 8 + 8
    assert ctypes.sizeof(lst.lst_launch) == 8 * 4


def test_ctypes_structs_match_the_c_header(tmp_path):
    """Every struct of include/lst.h, compiled by gcc: size and the offset of every field
    must equal the binding's ctypes layout."""
    from paper_2403_13166_gb300 import lst
    structs = {"lst_module": lst.lst_module, "lst_cuts": lst.lst_cuts, "lst_mlp": lst.lst_mlp,
               "lst_config": lst.lst_config, "lst_counts": lst.lst_counts, "lst_launch": lst.lst_launch,
               "lst_serve_config": lst.lst_serve_config, "lst_serve_result": lst.lst_serve_result,
               "lst_pixel_cuts": lst.lst_pixel_cuts, "lst_pixel_counts": lst.lst_pixel_counts}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "lst.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        sname, field, value = line.split()
        got[(sname, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_binding_constants_match_the_c_header(tmp_path):
    """Enum values and #define constants of include/lst.h, compiled by gcc, equal the
    binding's Python constants."""
    from paper_2403_13166_gb300 import lst
    names = {"LST_OK": lst.LST_OK, "LST_ERR_ARG": lst.LST_ERR_ARG, "LST_ERR_CAPACITY": lst.LST_ERR_CAPACITY,
             "LST_ERR_CUDA": lst.LST_ERR_CUDA, "LST_ERR_TIMEOUT": lst.LST_ERR_TIMEOUT,
             "LST_ERR_NOT_READY": lst.LST_ERR_NOT_READY, "LST_ERR_INPUT": lst.LST_ERR_INPUT,
             "LST_ERR_NOMEM": lst.LST_ERR_NOMEM, "LST_MD": lst.LST_MD, "LST_LS": lst.LST_LS,
             "LST_T3": lst.LST_T3, "LST_T5": lst.LST_T5, "LST_TC": lst.LST_TC, "LST_FP32": lst.LST_FP32,
             "LST_BF16": lst.LST_BF16, "LST_BF16X3": lst.LST_BF16X3, "LST_N_STAGES": lst.N_STAGES,
             "LST_GRAPH_NODE_FEATURES": lst.GRAPH_NODE_FEATURES,
             "LST_GRAPH_EDGE_FEATURES": lst.GRAPH_EDGE_FEATURES}
    lines = ['#include <stdio.h>', '#include "lst.h"', 'int main(void) {']
    lines += [f'  printf("{k} %d\\n", (int){k});' for k in names]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    got = dict(zip(out[::2], map(int, out[1::2])))
    assert got == names
    assert len(lst.STAGES) == lst.N_STAGES
