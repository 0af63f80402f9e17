"""Throughput benchmark of the LST hot path on PU200-like synthetic events.

One step = one batch of B PU200-like events (the workload of a single HL-LHC-like event,
many of them) through all stages: hit binning, mini-doublets, line segments, triplets,
quintuplets and the T5-DNN score. The headline `value` is the batched path (one
persistent launch per stage over the batch, replayed as a CUDA graph); `plain` is the
same events one launch sequence per event; `e2e` is the batched path through the C-ABI
with host (pinned) inputs and host outputs, copies inside the timed region.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU (torchrun): events are independent, every rank takes its own events (no data
exchange); only a barrier and a max over ranks of the elapsed time are collective.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PU200-like events/s on 1 GB300, plain vs batched+served; p50/p99 event latency"
PILEUP = 200
PER_VERTEX = 96          # particles per vertex: ~19k particles, ~250k hits per event
L2_BYTES = 129 * 2 ** 20


# ------------------------------------------------------------------ host-side workers (spawn)
def _gen_event(args):
    """(index, x, y, z, sensor, pixel seeds or None) of one synthetic event."""
    index, pileup, per_vertex, config = args[:4]
    with_seeds = len(args) > 4 and args[4]
    from paper_2403_13166_gb300 import synth
    g = _geom()
    e = synth.pileup_event(g, index, pileup=pileup, mean_per_vertex=per_vertex, config=config)
    return index, e.x, e.y, e.z, e.sensor, (synth.pixel_seeds(e).hits if with_seeds else None)


_GEOM = None


def _geom():
    global _GEOM
    if _GEOM is None:
        from paper_2403_13166_gb300 import synth
        _GEOM = synth.build_geometry(True)
    return _GEOM


def _oracle_time(args):
    """Oracle (as it stands) on one event; returns seconds of oracle time (generation excluded)."""
    index, pileup, per_vertex, config, weights, n_hidden, cut_set = args
    import oracle
    from paper_2403_13166_gb300 import synth
    g = _geom()
    e = synth.pileup_event(g, index, pileup=pileup, mean_per_vertex=per_vertex, config=config)
    cuts = _cut_set(cut_set)
    t0 = time.perf_counter()
    r = oracle.run_event(g, e, cuts, weights, n_hidden)
    dt = time.perf_counter() - t0
    return dt, r.counts["t5"]


# kernels of one launch sequence: reset, 3 grouping, 4 MD (grouping and order), 3 LS, 3 T3, T5,
# score, 4 track
# candidate, counter collection
KERNELS_PER_LAUNCH = 21

# score arithmetic of the batched and served forms (the plain form is always FP32)
PRECISIONS = {"fp32": 0, "bf16": 1, "bf16x3": 2}


def _cut_set(name):
    """'standard': the default cut parameters; 'open': the fit-quality tolerances of steps
    3-4 opened (the sample the T5-DNN is trained on, where it removes the fakes)."""
    from paper_2403_13166_gb300 import synth
    return synth.open_cuts() if name == "open" else synth.default_cuts()


def _weights():
    from paper_2403_13166_gb300 import synth, model_store
    w = model_store.load_trained()
    if w is not None:
        return w["flat"], w["n_hidden"], w.get("wp"), "trained"
    return synth.mlp_flat(synth.xavier_mlp()), 2, None, "xavier-seed2403"


def cpu_baseline(pool, n_cores, cut_set, events_per_core=2, config=2):
    """Bounded sample: every core runs `events_per_core` oracle events (~1 s each)."""
    flat, nh, _, _ = _weights()
    jobs = [(10_000 + i, PILEUP, PER_VERTEX, config, flat, nh, cut_set) for i in range(n_cores * events_per_core)]
    t0 = time.perf_counter()
    res = pool.map(_oracle_time, jobs, chunksize=events_per_core)
    wall = time.perf_counter() - t0
    times = [r[0] for r in res]
    # per-core sums -> throughput with all cores busy, excluding the generator's time
    per_core = [sum(times[i::n_cores]) for i in range(n_cores)]
    value = len(times) / max(per_core)
    return {"value": round(value, 3), "unit": "events/s", "cores": n_cores, "kind": "oracle",
            "sample": f"{len(times)} PU200-like events ({events_per_core} per core, oracle time only, "
                      f"{sum(times):.1f} s CPU, generation excluded)",
            "value_1core": round(1.0 / statistics.mean(times), 3), "wall_s": round(wall, 2)}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", self.gpu_id], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            time.sleep(0.15)
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        sm, mx, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def nvsmi_index(torch, dev, local_rank) -> str:
    """nvidia-smi index of the torch device (matched by UUID), else the visible index."""
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid).lower()
        out = subprocess.run(["nvidia-smi", "--query-gpu=index,uuid", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            i, uu = [x.strip() for x in line.split(",")]
            if u and u in uu.lower():
                return i
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[local_rank].strip().isdigit():
        return vis.split(",")[local_rank].strip()
    return str(local_rank)


# ------------------------------------------------------------------ multi-rank host logic
def rank_event_indices(rank: int, batch: int):
    """Event seeds of one rank: disjoint across ranks (events are independent units)."""
    return [rank * 100_000 + i for i in range(batch)]


def max_over_ranks(x: float, device) -> float:
    """Slowest rank's elapsed time: the only collective of the benchmark."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(events_per_rank: int, world: int, seconds_max: float) -> float:
    """Events of all ranks divided by the slowest rank's time."""
    return events_per_rank * world / seconds_max


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world, local_rank, pool):
    import torch
    from paper_2403_13166_gb300 import lst, synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    B = args.batch
    # events of this rank (distinct seeds per rank)
    idx = rank_event_indices(rank, B)
    evs = pool.map(_gen_event, [(i, PILEUP, PER_VERTEX, 2, not args.skip_plain) for i in idx])
    n_hits = np.array([len(e[1]) for e in evs])
    g = _geom()
    flat, nh, wp, wname = _weights()
    cuts = _cut_set(args.cuts)
    if wp is not None:
        cuts["wp"] = np.float32(wp)
    precision = PRECISIONS[args.precision]
    ctx = lst.Context(local_rank, max_events=3 * B, precision=precision, use_graphs=1)
    ctx.load_geometry(g, cuts, flat, nh)
    # the plain form: one launch sequence per event, FP32 score
    ctx_p = lst.Context(local_rank, max_events=2, precision=lst.LST_FP32, use_graphs=0)
    ctx_p.load_geometry(g, cuts, flat, nh)
    d_in = [[torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in e[1:5]] for e in evs]
    stream = torch.cuda.current_stream(dev)
    tuned = None
    if args.tune:   # launch shapes from the project's autotuner (tuned once per GPU and workload)
        from paper_2403_13166_gb300 import autotune
        tuned = autotune.tune_or_load(ctx, d_in, device=local_rank, stream=stream)

    def sync_all():
        torch.cuda.synchronize(dev)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # three batches in flight: each step enqueues one and then takes the results of the one
    # launched two steps before, so a late host leaves the GPU a whole batch of work
    def batched_step(inputs, pending):
        pending = (pending or []) + [ctx.run_batch(inputs, stream)]
        if len(pending) > 2:
            for h in pending.pop(0):
                c = h.counts()
                if c["status"] != lst.LST_OK:
                    raise RuntimeError(f"event status {c['status']}")
                h.release()
        return pending

    def drain(pending):
        out = []
        for hs in pending or []:
            out = []
            for h in hs:
                out.append(h.counts())
                h.release()
        return out

    # ---------------- batched (graph) path; warm-up captures the same (timed) graph
    ctx.set_timing(True)
    prev = None
    for _ in range(args.warmup):
        prev = batched_step(d_in, prev)
    counts = drain(prev)
    prev = None
    ctx.set_timing(True)   # resets the stage statistics
    gpu_id = nvsmi_index(torch, dev, local_rank)
    sync_all()
    with ClockSampler(gpu_id) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            prev = batched_step(d_in, prev)
        drain(prev)
        e1.record(stream)
        sync_all()
    ms_total = e0.elapsed_time(e1)
    stage_ms, n_launch = ctx.stage_times()
    ctx.set_timing(False)
    if world > 1:
        import torch.distributed as dist
        ms_total = max_over_ranks(ms_total, dev)
    value = whole_job_rate(B * args.steps, world, ms_total / 1000.0)

    # ---------------- plain path: one launch sequence per event
    plain = None
    if not args.skip_plain:
        n_plain = min(B, args.plain_events)
        for i in range(min(3, n_plain)):
            ctx_p.run_event(*d_in[i], stream=stream).release()
        sync_all()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for i in range(n_plain):
            ctx_p.run_event(*d_in[i], stream=stream).release()
        p1.record(stream)
        sync_all()
        pms = p0.elapsed_time(p1)
        plain = {"value": round(n_plain / (pms / 1000.0), 2), "unit": "events/s",
                 "ms_per_event": round(pms / n_plain, 4), "events": n_plain, "score_precision": "fp32",
                 "gpu_launches_per_event": KERNELS_PER_LAUNCH, "form": "one launch sequence per event, no graph"}

    # ---------------- LS graph (Section 4): MD nodes, LS edges, exported as CSR on the device
    graph = None
    if not args.skip_plain:
        caps = int(3 * max(n_hits)), int(20 * max(n_hits))
        g_row = torch.empty(caps[0] + 1, dtype=torch.int32, device=dev)
        g_col = torch.empty(caps[1], dtype=torch.int32, device=dev)
        g_nf = torch.empty((caps[0], lst.GRAPH_NODE_FEATURES), dtype=torch.float32, device=dev)
        g_ef = torch.empty((caps[1], lst.GRAPH_EDGE_FEATURES), dtype=torch.float32, device=dev)
        times, sizes = [], []
        for i in range(min(8, B)):
            ev = ctx_p.run_event(*d_in[i], stream=stream)
            sync_all()
            t0 = time.perf_counter()
            sizes.append(ev.ls_graph_into(g_row, g_col, g_nf, g_ef))
            times.append(time.perf_counter() - t0)
            ev.release()
        graph = {"export_ms_per_event": round(1000 * float(np.median(times[1:] or times)), 4),
                 "nodes_per_event": int(np.mean([s[0] for s in sizes])),
                 "edges_per_event": int(np.mean([s[1] for s in sizes]))}

    # ---------------- pixel seeds (Table 1 steps 5-8): pT5 / T5 / pT3 / pLS track candidates
    # (seeds from each event's particles, made with the event); all events of the batch in
    # one call, and one event per call for comparison
    pixel = None
    if not args.skip_plain:
        pcuts = synth.default_pixel_cuts()
        seeds = [torch.from_numpy(e[5]).to(dev) for e in evs]
        hs = ctx.run_batch(d_in, stream)
        for h in hs:
            h.counts()
        ctx.match_pixel_seeds_batch(hs, seeds, pcuts)          # buffers sized once
        sync_all()
        t0 = time.perf_counter()
        cnts = ctx.match_pixel_seeds_batch(hs, seeds, pcuts)
        t_batch = time.perf_counter() - t0
        single = []
        for i in range(min(5, B)):
            t0 = time.perf_counter()
            hs[i].match_pixel_seeds(seeds[i], pcuts)
            single.append(time.perf_counter() - t0)
        for h in hs:
            h.release()
        pixel = {"match_ms_per_event": round(1000 * t_batch / B, 4),
                 "form": f"all {B} events in one call (lst_match_pixel_seeds_batch), device seeds, synchronous",
                 "match_ms_per_event_single_call": round(1000 * float(np.median(single)), 4),
                 "per_event_mean": {k: round(float(np.mean([c[k] for c in cnts])), 1)
                                    for k in ("n_pt5", "n_t5", "n_pt3", "n_pls", "rounds_pt5", "rounds_pt3")}}

    # ---------------- e2e: host pinned inputs -> C-ABI -> host outputs (T5 tuples + scores)
    pinned = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in e[1:5]] for e in evs]
    h2d = int(sum(16 * n for n in n_hits))
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    # pinned result buffers for the whole batch (one export call per step)
    cap5 = int(1.5 * B * max(c["t5"] for c in counts)) + 1024
    r_hits = torch.empty((cap5, 10), dtype=torch.int32).pin_memory().numpy()
    r_score = torch.empty(cap5, dtype=torch.float32).pin_memory().numpy()
    r_sel = torch.empty(cap5, dtype=torch.uint8).pin_memory().numpy()

    def export(hs):
        _, _, _, offs = ctx.candidates_batch(hs, lst.LST_T5, r_hits, r_score, r_sel)
        for h in hs:
            h.release()
        return int(offs[-1]) * (40 + 4 + 1) + 8 * (B + 1)

    # three streams in turn, so that the host-to-device copies of the next batches overlap
    # the kernels of the current one
    e2e_streams = [stream, torch.cuda.Stream(dev), torch.cuda.Stream(dev)]

    def e2e_run(steps):
        # batches k+1 and k+2 are enqueued (H2D + kernels) before batch k's results are read
        # back (three batches in flight, as in the device-resident loop)
        pending, d2h = [], 0
        for k in range(steps):
            pending.append(ctx.run_batch(pinned, e2e_streams[k % 3]))
            if len(pending) > 2:
                d2h += export(pending.pop(0))
        for hs in pending:
            d2h += export(hs)
        return d2h

    e2e_run(3)
    sync_all()
    t0 = time.perf_counter()
    d2h = e2e_run(e2e_steps)
    sync_all()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        import torch.distributed as dist
        e2e_s = max_over_ranks(e2e_s, dev)
    e2e = {"value": round(B * e2e_steps * world / e2e_s, 2), "unit": "events/s",
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(d2h / e2e_steps),
           "steps": e2e_steps}

    # ---------------- served: Poisson arrivals, continuous batching, tensor-core score
    served = None
    if not args.skip_served and world == 1:
        served = run_served(args, pool, g, cuts, flat, nh, local_rank)

    # ---------------- roofline of the dominant kernel
    c0 = counts[0] if counts else {}
    mean_counts = {k: float(np.mean([c[k] for c in counts])) for k in ("md", "ls", "t3", "t5")}
    pairs = np.mean(np.array([c["pairs"] for c in counts], np.float64), axis=0)
    names = list(lst.STAGES)
    dom = int(np.argmax(stage_ms))
    roofline = roofline_entry(names[dom], float(stage_ms[dom]), B, mean_counts, pairs, float(np.mean(n_hits)),
                              clk.summary(), torch.cuda.get_device_properties(dev).multi_processor_count)
    roofline["stage_ms_per_launch"] = {n: round(float(v), 4) for n, v in zip(names, stage_ms)}
    step = step_roofline(mean_counts, pairs, float(np.mean(n_hits)), float(np.mean(np.diff(g.map_off))),
                         value, clk.summary(), torch.cuda.get_device_properties(dev).multi_processor_count)
    score_rf = score_roofline(float(stage_ms[names.index("score")]), B, mean_counts, precision)
    if graph is not None:   # the graph build inside the batched launch: grouping, MD and LS stages
        graph["build_ms_per_event_batched"] = round(float(sum(stage_ms[:4])) / B, 4)
    roofline["launches_timed"] = int(n_launch)

    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "events/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_total / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if precision == lst.LST_FP32 else "f32+bf16",
        "data": "synthetic",
        "config": {"workload": "pu200_like_batched", "events_per_step": B, "pileup": PILEUP,
                   "particles_per_vertex": PER_VERTEX, "hits_per_event_mean": int(np.mean(n_hits)),
                   "modules": g.n_mod, "score_precision": args.precision, "weights": wname, "cuts": args.cuts,
                   "graphs": True, "l2": f"inputs larger than L2 ({int(h2d / 2**20)} MiB of hits per step)",
                   "launch": ctx.get_launch(), "autotuned": None if tuned is None else
                   {"cached": tuned["cached"], "trials": len(tuned.get("trials", []))},
                   "objects_per_event_mean": {k: int(v) for k, v in mean_counts.items()}},
        "plain": plain,
        "served": served,
        "ls_graph": graph,
        "pixel_tc": pixel,
        "e2e": e2e,
        "roofline": roofline,
        "step_roofline": step,
        "score_roofline": score_rf,
        "clocks": clk.summary(),
        "gpu_launches": KERNELS_PER_LAUNCH * args.steps,
    }
    ctx.close()
    ctx_p.close()
    return line


def run_served(args, pool, g, cuts, flat, nh, local_rank):
    """Requests arrive one at a time (Poisson) and are served by the library's continuous-
    batching worker; latency = completion of the event (results on the host) - arrival."""
    import torch
    from paper_2403_13166_gb300 import lst
    rng = np.random.default_rng(5)
    pus = rng.integers(140, 201, args.served_pool)
    evs = pool.map(_gen_event, [(500_000 + i, int(pu), PER_VERTEX, 5) for i, pu in enumerate(pus)])
    pinned = [[torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in e[1:5]] for e in evs]
    ctx = lst.Context(local_rank, max_events=2 * args.batch, precision=PRECISIONS[args.precision], use_graphs=1)
    ctx.load_geometry(g, cuts, flat, nh)
    out = {"workload": "pu140_200_poisson", "pool_events": int(args.served_pool), "max_batch": args.served_max_batch,
           "lanes": 2, "score_precision": args.precision, "rates": []}
    # the batched rate on the same pool (device inputs, batches of args.batch pool events, two
    # in flight): what the served rates are compared with
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    d_pool = [[torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in e] for e in pinned]
    batch_in = [d_pool[k % len(d_pool)] for k in range(args.batch)]

    def step(prev):
        hs = ctx.run_batch(batch_in, stream)
        for h in prev or []:
            h.release()
        return hs
    prev = None
    for _ in range(3):
        prev = step(prev)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        prev = step(prev)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    for h in prev:
        h.release()
    out["batched_same_pool_per_s"] = round(10 * args.batch / (e0.elapsed_time(e1) / 1000.0), 1)
    del d_pool, batch_in
    slot_hits = int(1.2 * max(len(e[0]) for e in pinned))     # every slot sized for the pool's events
    srv = lst.Server(ctx, max_batch=args.served_max_batch, lanes=2, mem_budget_bytes=int(args.served_mem_gb * 2**30),
                     copy_t5=True, slot_hits=slot_hits)
    # warm-up: one burst (captures the graphs for the batch sizes seen first)
    for k in range(2 * args.batch):
        e = pinned[k % len(pinned)]
        srv.submit(*e, tag=k)
    got = 0
    while got < 2 * args.batch:
        got += len(srv.poll(wait_ms=100, keep_t5=False))
    tag = 10**6
    import gc
    for rate in args.served_rates:
        # no garbage-collection pause of this client inside a rate's window (arrival times are
        # the scheduled ones, so a stalled client would show as server latency)
        gc.collect()
        gc.disable()
        n = max(50, int(rate * args.served_seconds))
        gaps = rng.exponential(1.0 / rate, n)
        t0 = lst.clock() + 0.01
        arr = t0 + np.cumsum(gaps)
        res = []
        for k in range(n):
            while True:
                now = lst.clock()
                if now >= arr[k]:
                    break
                if arr[k] - now > 0.002:
                    time.sleep(0.0005)
                res.extend(srv.poll(keep_t5=False))
            e = pinned[k % len(pinned)]
            srv.submit(*e, tag=tag + k, t_arrival=float(arr[k]))
        while len(res) < n:
            res.extend(srv.poll(wait_ms=100, keep_t5=False))
        gc.enable()
        tag += n
        lat = np.array([r["t_done"] - r["t_arrival"] for r in res]) * 1000.0
        ok = all(r["status"] == lst.LST_OK for r in res)
        span = max(r["t_done"] for r in res) - arr[0]
        # steady state: completions between the 10th and the 90th percentile of completion
        # time over that interval (the fill at the start and the drain after the last
        # arrival, ~one latency long, do not count)
        td = np.sort([r["t_done"] for r in res])
        k0, k1 = n // 10, n - 1 - n // 10
        sustained = (k1 - k0) / max(td[k1] - td[k0], 1e-9)
        out["rates"].append({"offered_per_s": rate, "events": n, "achieved_per_s": round(n / span, 1),
                             "sustained_per_s": round(float(sustained), 1),
                             "p50_ms": round(float(np.percentile(lat, 50)), 3),
                             "p99_ms": round(float(np.percentile(lat, 99)), 3), "all_ok": ok})
    srv.stop()
    ctx.close()
    return out


# Algorithmic work for the roofline: FP32 operations of the full cut expression tree per
# candidate pair of each step (the specification's per-unit figures: MD 25, LS 45, T3 40,
# T5 70). The strict alternative counts only the z0 test every LS pair needs (12) plus the
# rest of the cut per accepted LS (35); it is reported beside as `achieved_strict`.
FP32_OPS_PER_PAIR = {"md": 25, "ls": 45, "t3": 40, "t5": 70}
STRICT_OPS = {"ls": (12, 35)}


# DRAM bytes (read + write) per event of a kernel, from one ncu capture of a 16-event
# launch of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum = 65.38 +
# 244.44 MB for k_ls); the traffic is the per-event LS output plus MD reads, so it scales
# with the events.
TRAFFIC_PER_EVENT = {"ls": 309.82e6 / 16}


def traffic_per_launch(stage, events):
    b = TRAFFIC_PER_EVENT.get(stage)
    return None if b is None else int(b * events)


def roofline_entry(stage, ms, B, counts, pairs, hits, clocks, n_sm):
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    if stage in ("md", "ls", "t3", "t5"):
        k = ["md", "ls", "t3", "t5"].index(stage)
        ops = B * pairs[k] * FP32_OPS_PER_PAIR[stage]
        sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12       # FP32 peak, an FMA counted as 2
        issue = peak / 2                                   # one FP32 operation per lane per clock
        achieved = ops / (ms / 1000.0) / 1e12
        out = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
               "frac": round(achieved / peak, 4), "traffic": traffic_per_launch(stage, B), "kernel": f"k_{stage}",
               "peak_note": f"FP32 peak: {n_sm} SMs x 128 lanes x 2 (FMA) x {sm_mhz:.0f} MHz (SM clock "
                            f"sampled during the timed region)",
               "peak_issue": round(issue, 2), "frac_issue": round(achieved / issue, 4),
               "issue_note": "the cut code may not contract a*b+c (bit-exact FP32 parity), so one FP32 "
                             "operation per lane per clock is its ceiling",
               "ops_per_pair": FP32_OPS_PER_PAIR[stage]}
        if stage in STRICT_OPS:
            a, b = STRICT_OPS[stage]
            strict = B * (pairs[k] * a + counts[stage] * b) / (ms / 1000.0) / 1e12
            out["achieved_strict"] = round(strict, 3)
            out["frac_strict"] = round(strict / peak, 4)
            out["frac_strict_issue"] = round(strict / issue, 4)
        return out
    # score / bin: HBM bound
    hbm = peaks.get("hbm_gbs", 6800.0)
    if stage == "score":
        by = B * counts["t5"] * (32 + 5 * (16 + 8 + 4) + 5)
    else:
        by = B * hits * (16 + 20 + 20)
    achieved = by / (ms / 1000.0) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": None, "kernel": f"k_{stage}",
            "peak_note": "measured" if peaks else "fallback"}


# Whole-step algorithmic work per event (every object read once per consuming stage and
# written once; MDs read once as inner and once per module-map link as targets), and FP32
# operations of the cut expression trees per candidate pair plus the network per T5.
STEP_OPS_PER_PAIR = (25, 45, 40, 70)     # MD, LS, T3, T5
MLP_FLOP_PER_T5 = 4544


def step_roofline(counts, pairs, hits, fan, events_per_s, clocks, n_sm):
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    by = (hits * (16 + 20 + 20) + counts["md"] * (28 + 28 * (1 + fan)) + counts["ls"] * (12 + 24)
          + counts["t3"] * (12 + 24) + counts["t5"] * (20 + 5 * 16 + 5))
    ops = sum(float(p) * k for p, k in zip(pairs, STEP_OPS_PER_PAIR)) + MLP_FLOP_PER_T5 * counts["t5"]
    hbm = peaks.get("hbm_gbs", 6800.0)
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    alu = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    gbs = by * events_per_s / 1e9
    tops = ops * events_per_s / 1e12
    return {"alg_bytes_per_event": int(by), "alg_fp32_ops_per_event": int(ops),
            "achieved_GBs": round(gbs, 1), "hbm_peak_GBs": hbm, "hbm_frac": round(gbs / hbm, 4),
            "achieved_TOPs": round(tops, 3), "alu_peak_TOPs": round(alu, 2), "alu_frac": round(tops / alu, 4),
            "alu_issue_frac": round(2 * tops / alu, 4),
            "note": "mean module-map fan-out %.1f; FP32 ops per candidate pair MD/LS/T3/T5 = %s" % (
                fan, "/".join(map(str, STEP_OPS_PER_PAIR)))}


def score_roofline(ms, B, counts, precision):
    """The T5-DNN stage against the tensor peak (the network's 4544 flop per T5; the split
    form issues three MMAs per K-step) and against HBM (what the feature gather reads)."""
    from paper_2403_13166_gb300 import lst
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    t5 = B * counts["t5"]
    sec = ms / 1000.0
    flop = t5 * MLP_FLOP_PER_T5
    by = t5 * (32 + 5 * (16 + 8 + 4) + 5)
    hbm = peaks.get("hbm_gbs", 6800.0)
    out = {"stage_ms_per_launch": round(ms, 4), "t5_per_launch": int(t5),
           "hbm_achieved_GBs": round(by / sec / 1e9, 1), "hbm_frac": round(by / sec / 1e9 / hbm, 4)}
    if precision == lst.LST_FP32:
        out.update({"kernel": "k_score_fp32", "bound": "alu", "achieved": round(flop / sec / 1e12, 3),
                    "unit": "TFLOP/s", "note": "compensated FP32 (float-float) layers on the CUDA cores"})
        return out
    mma = 3 if precision == lst.LST_BF16X3 else 1
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    achieved = flop / sec / 1e12
    out.update({"kernel": "k_score_bf16", "bound": "tensor", "achieved": round(achieved, 3), "peak": peak,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 5), "mma_per_kstep": mma,
                "issued_frac": round(mma * achieved / peak, 5),
                "peak_note": ("measured sustained bf16 (cuBLAS)" if peaks else "fallback"),
                "note": "the stage gathers each T5's features from five MD anchors; the tensor pipe "
                        "is idle most of the time (feature gathering bounds it)"})
    return out


# ------------------------------------------------------------------ reference arm: the oracle
def run_reference(args, pool, n_cores):
    flat, nh, _, _ = _weights()
    per_step = n_cores          # one event per core per step (~1 s of oracle work each)
    jobs = lambda s: [(20_000 + s * per_step + i, PILEUP, PER_VERTEX, 2, flat, nh, args.cuts)
                      for i in range(per_step)]
    for s in range(args.warmup):
        pool.map(_oracle_time, jobs(s), chunksize=1)
    busy = []
    t0 = time.perf_counter()
    for s in range(args.steps):
        res = pool.map(_oracle_time, jobs(args.warmup + s), chunksize=1)
        busy.append(max(r[0] for r in res))
    wall = time.perf_counter() - t0
    oracle_s = sum(busy)
    value = per_step * args.steps / oracle_s
    return {"metric": METRIC, "value": round(value, 3), "unit": "events/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * oracle_s / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "impl": "reference", "hardware": f"{n_cores} host cores, no GPU",
            "config": {"workload": "pu200_like_batched", "events_per_step": per_step, "pileup": PILEUP,
                       "particles_per_vertex": PER_VERTEX, "cuts": args.cuts},
            "cpu_baseline": {"value": round(value, 3), "unit": "events/s", "cores": n_cores, "kind": "oracle",
                             "sample": f"{per_step} PU200-like events per step, one per core, oracle time "
                                       f"only (generation excluded); wall {wall:.1f} s"},
            "e2e": {"value": round(value, 3), "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="lst", choices=["lst", "reference"])
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--precision", default="bf16x3", choices=list(PRECISIONS))
    ap.add_argument("--plain-events", type=int, default=64)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="skip the launch-shape autotuner (default: tune once per GPU and workload)")
    ap.add_argument("--skip-served", action="store_true")
    ap.add_argument("--served-rates", type=float, nargs="+", default=[100, 500, 1000, 2000, 3000, 4000, 5000, 6000, 7000])
    ap.add_argument("--served-seconds", type=float, default=3.0)
    ap.add_argument("--served-pool", type=int, default=48)
    ap.add_argument("--served-mem-gb", type=float, default=16.0)
    ap.add_argument("--served-max-batch", type=int, default=64, help="largest batch of one served launch")
    ap.add_argument("--cuts", default="standard", choices=["standard", "open"])
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    n_cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    # the process pool starts with `spawn` before any GPU call
    ctx_mp = mp.get_context("spawn")
    if args.impl == "reference":
        if rank != 0:
            return
        with ctx_mp.Pool(n_cores) as pool:
            print(json.dumps(run_reference(args, pool, n_cores)), flush=True)
        return
    with ctx_mp.Pool(min(n_cores, 16)) as pool:
        cpu = None
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline(pool, min(n_cores, 16), args.cuts)
        if world > 1:
            import torch.distributed as dist
            import torch
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        line = run_gpu(args, rank, world, local_rank, pool)
        line["cpu_baseline"] = cpu
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
