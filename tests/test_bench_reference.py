"""bench.py --impl reference (the oracle on the host cores) prints one JSON line with the
benchmark contract's keys, the same metric and unit as the GPU arm, and a cpu_baseline
describing its own run. CPU only (a short run: one timed step of one event per core)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    sys.path.insert(0, ROOT)
    import bench
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "events/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3 and d["value"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "pu200_like_batched"


def test_roofline_fields_follow_their_definitions():
    """The bench line's roofline objects, from fixed inputs: achieved = the specification's
    work / time, frac = achieved / peak; the FP32 peak counts an FMA as two operations and
    the issue peak is half of it; the score stage is measured against the tensor peak, with
    the split form issuing three MMAs per K-step."""
    sys.path.insert(0, ROOT)
    import bench
    pairs = [3.41e6, 59.3e6, 5.91e6, 51.6e3]
    counts = {"md": 1.18e5, "ls": 1.11e6, "t3": 1.13e5, "t5": 4.25e4}
    clocks = {"sm_mhz": 2000.0}
    r = bench.roofline_entry("ls", 5.0, 64, counts, pairs, 2.5e5, clocks, 152)
    peak = 152 * 128 * 2 * 2000e6 / 1e12
    achieved = 64 * 59.3e6 * 45 / 5e-3 / 1e12
    assert abs(r["peak"] - round(peak, 2)) < 1e-9 and abs(r["peak_issue"] - round(peak / 2, 2)) < 1e-9
    assert abs(r["achieved"] - achieved) < 1e-3 and abs(r["frac"] - achieved / peak) < 1e-4
    assert abs(r["frac_issue"] - 2 * achieved / peak) < 1e-4 and r["bound"] == "alu"
    strict = 64 * (59.3e6 * 12 + 1.11e6 * 35) / 5e-3 / 1e12
    assert abs(r["achieved_strict"] - strict) < 1e-3
    from paper_2403_13166_gb300 import lst
    s1 = bench.score_roofline(0.5, 64, counts, lst.LST_BF16)
    s3 = bench.score_roofline(0.5, 64, counts, lst.LST_BF16X3)
    flop = 64 * 4.25e4 * bench.MLP_FLOP_PER_T5 / 5e-4 / 1e12
    assert s1["bound"] == "tensor" and abs(s1["achieved"] - flop) < 1e-3
    assert s1["mma_per_kstep"] == 1 and s3["mma_per_kstep"] == 3
    assert abs(s3["issued_frac"] - 3 * s3["frac"]) < 1e-4 and abs(s1["frac"] - flop / s1["peak"]) < 1e-4
    assert bench.score_roofline(0.5, 64, counts, lst.LST_FP32)["bound"] == "alu"
