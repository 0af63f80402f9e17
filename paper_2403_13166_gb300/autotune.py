"""Launch-shape autotuner for the batched pipeline.

Each tunable of lst_launch belongs to one stage (CTA sizes of steps 1-4 and of the FP32
score), and the library times every
stage separately (lst_stage_times, CUDA events inside the launch). The tuner therefore
does coordinate descent: for one parameter at a time it replays the caller's own batch
with every candidate value and keeps the value whose stage time is lowest (by more than
`min_gain`), every other parameter fixed. Each trial must reproduce the object counts of
the starting shape exactly: a launch shape changes how work is distributed, never what
is found, and the tuner refuses a shape that breaks that.

Results are cached per GPU (name, SM count) and workload (batch size, mean hits per event
rounded to 10k) in a JSON file:

    from paper_2403_13166_gb300 import autotune
    shape = autotune.tune_or_load(ctx, device_inputs)     # tunes once, then reuses
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import lst

SPACE = {
    "ls_threads": (64, 96, 128, 160, 192, 256),
    "md_threads": (64, 128, 192, 256),
    "t3_threads": (64, 128, 192, 256),
    "t5_threads": (64, 128, 256),
    "sc_threads": (128, 256),
}
# ls_list is unused by the library (kept in lst_launch for layout); listed so that an
# explicit space may still name it
STAGE = {"md_threads": 1, "ls_threads": 2, "ls_list": 2, "t3_threads": 4, "t5_threads": 5, "sc_threads": 6}
COUNT_KEYS = ("md", "ls", "t3", "t5", "tc", "selected")
CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_tuned", "launch_cache.json")


def _device_key(device: int) -> str:
    import torch
    p = torch.cuda.get_device_properties(device)
    return f"{p.name}|sm{p.multi_processor_count}"


def workload_key(inputs) -> str:
    hits = float(np.mean([int(t[0].shape[0]) for t in inputs])) if inputs else 0.0
    return f"batch{len(inputs)}|hits{int(round(hits, -4))}"


def _measure(ctx, inputs, reps, stream):
    hs = ctx.run_batch(inputs, stream)           # first run: graph capture, warm caches
    for h in hs:
        h.release()
    ctx.set_timing(True)
    counts = None
    for _ in range(reps):
        hs = ctx.run_batch(inputs, stream)
        c = [h.counts() for h in hs]
        for h in hs:
            h.release()
        counts = counts or c
    ms, _ = ctx.stage_times()
    ctx.set_timing(False)
    for c in counts:
        if c["status"] != lst.LST_OK:
            raise RuntimeError(f"event status {c['status']} during tuning")
    return ms, [tuple(c[k] for k in COUNT_KEYS) + tuple(c["pairs"]) for c in counts]


def tune(ctx, inputs, reps: int = 3, stream=None, space=None, min_gain: float = 0.02, log=None) -> dict:
    """Coordinate descent over `space` (default SPACE) on the batch `inputs` (device
    tensors, as for Context.run_batch). Leaves the best shape set on ctx and returns it."""
    space = SPACE if space is None else space
    best = ctx.get_launch()
    ms, ref = _measure(ctx, inputs, reps, stream)
    stage_ms = list(ms)
    trials = []
    for param, values in space.items():
        k = STAGE[param]
        for v in values:
            if v == best[param]:
                continue
            trial = dict(best, **{param: v})
            try:
                ctx.set_launch(**trial)
            except lst.LstError:
                continue                          # e.g. the shared memory of the shape is too large
            t_ms, got = _measure(ctx, inputs, reps, stream)
            if got != ref:
                raise RuntimeError(f"launch shape {trial} changed the results")
            trials.append({"param": param, "value": v, "stage_ms": float(t_ms[k])})
            if log:
                log(f"{param}={v}: stage {lst.STAGES[k]} {t_ms[k]:.3f} ms (best {stage_ms[k]:.3f})")
            if t_ms[k] < stage_ms[k] * (1.0 - min_gain):
                best, stage_ms = trial, list(t_ms)
        ctx.set_launch(**best)
    return {"launch": best, "stage_ms": [float(x) for x in stage_ms], "trials": trials}


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def apply_cached(ctx, inputs, device: int = 0, path: str = CACHE) -> dict | None:
    """Set the cached shape for this GPU and workload on ctx; None when there is none."""
    entry = _load_cache(path).get(_device_key(device) + "|" + workload_key(inputs))
    if entry is None:
        return None
    ctx.set_launch(**entry["launch"])
    return entry


def tune_or_load(ctx, inputs, device: int = 0, path: str = CACHE, **kw) -> dict:
    entry = apply_cached(ctx, inputs, device, path)
    if entry is not None:
        return dict(entry, cached=True)
    entry = tune(ctx, inputs, **kw)
    cache = _load_cache(path)
    cache[_device_key(device) + "|" + workload_key(inputs)] = {"launch": entry["launch"],
                                                                "stage_ms": entry["stage_ms"]}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return dict(entry, cached=False)
