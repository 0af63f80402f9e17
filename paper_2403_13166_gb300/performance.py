"""Tracking performance of the track candidates on synthetic truth (the metrics of
Sections 1 and 3): efficiency = fraction of findable simulated particles matched by at least
one track candidate (> 75% of its hits from the particle); fake rate = fraction of track
candidates matched to no particle; duplicate rate = fraction of found particles matched
by more than one. Efficiency is binned in the particle's pT, eta and transverse
production radius r_vertex; fake rate in the candidate's own pT and eta (from the circle
through its first, middle and last anchor and the chord's slope in r-z).

The comparison of Section 3 (pre-DNN vs T5-DNN at equal efficiency) runs as

    python -m paper_2403_13166_gb300.performance --sample pu200 --events 20 --out perf.json

on the library: the DNN mode with the trained network, the pre-DNN mode (circle-fit chi2
selection), and the DNN mode with its working point moved until its efficiency matches
the pre-DNN mode's (bisection on the working point, one library run per step)."""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import synth, truth

PT_BINS = np.array([0.8, 1.0, 1.5, 2.0, 3.0, 5.0, 10.0, 1e9])
ETA_BINS = np.linspace(-2.4, 2.4, 13)
RV_BINS = np.array([0.0, 0.1, 1.0, 2.0, 3.0, 5.0, 7.5, 10.0, 1e9])


def candidate_kinematics(tc_hits: np.ndarray, e) -> tuple[np.ndarray, np.ndarray]:
    """(pT, eta) of each candidate from its lower-sensor hits (anchors) 0, 2 and 4, FP64."""
    if len(tc_hits) == 0:
        return np.zeros(0), np.zeros(0)
    a = tc_hits[:, 0::2]
    x, y, z = (np.asarray(v, np.float64)[a] for v in (e.x, e.y, e.z))
    ax, ay = x[:, 2] - x[:, 0], y[:, 2] - y[:, 0]
    bx, by = x[:, 4] - x[:, 2], y[:, 4] - y[:, 2]
    cx, cy = x[:, 4] - x[:, 0], y[:, 4] - y[:, 0]
    cross = ax * cy - ay * cx
    abc = np.hypot(ax, ay) * np.hypot(bx, by) * np.hypot(cx, cy)
    kappa = np.abs(2.0 * cross / np.where(abc > 0, abc, np.inf))
    pt = synth.K_FIELD / np.maximum(kappa, 1e-9)
    r = np.hypot(x, y)
    eta = np.arcsinh((z[:, 4] - z[:, 0]) / np.maximum(r[:, 4] - r[:, 0], 1e-9))
    return pt, eta


class Tally:
    """Counts accumulated over events; ratios on demand."""

    def __init__(self):
        self.found = {k: np.zeros(len(b) - 1) for k, b in (("pt", PT_BINS), ("eta", ETA_BINS), ("rv", RV_BINS))}
        self.denom = {k: np.zeros_like(v) for k, v in self.found.items()}
        self.fake = {k: np.zeros(len(b) - 1) for k, b in (("pt", PT_BINS), ("eta", ETA_BINS))}
        self.cands = {k: np.zeros_like(v) for k, v in self.fake.items()}
        self.n_findable = self.n_found = self.n_dup = self.n_tc = self.n_fake = 0

    def add(self, tc_hits: np.ndarray, e, layer_of_module: np.ndarray):
        P = e.particles
        n_part = len(P["pt"])
        m = truth.match_particle(tc_hits, e.pid)
        per = np.bincount(m[m >= 0], minlength=n_part) if n_part else np.zeros(0, np.int64)
        fnd = truth.findable_t5(e.sensor, e.pid, layer_of_module, n_part)
        hit = per[fnd] > 0
        self.n_findable += len(fnd)
        self.n_found += int(hit.sum())
        self.n_dup += int((per[fnd] > 1).sum())
        var = {"pt": P["pt"][fnd], "eta": P["eta"][fnd], "rv": np.hypot(P["vx"], P["vy"])[fnd]}
        for k, b in (("pt", PT_BINS), ("eta", ETA_BINS), ("rv", RV_BINS)):
            self.denom[k] += np.histogram(var[k], b)[0]
            self.found[k] += np.histogram(var[k][hit], b)[0]
        pt, eta = candidate_kinematics(tc_hits, e)
        fake = m < 0
        self.n_tc += len(m)
        self.n_fake += int(fake.sum())
        for k, v, b in (("pt", pt, PT_BINS), ("eta", eta, ETA_BINS)):
            self.cands[k] += np.histogram(v, b)[0]
            self.fake[k] += np.histogram(v[fake], b)[0]

    def result(self) -> dict:
        def ratio(a, b):
            return [round(float(x / y), 5) if y else None for x, y in zip(a, b)]
        return {
            "efficiency": self.n_found / max(1, self.n_findable),
            "fake_rate": self.n_fake / max(1, self.n_tc),
            "duplicate_rate": self.n_dup / max(1, self.n_found),
            "findable": self.n_findable, "track_candidates": self.n_tc,
            "efficiency_vs_pt": ratio(self.found["pt"], self.denom["pt"]),
            "efficiency_vs_eta": ratio(self.found["eta"], self.denom["eta"]),
            "efficiency_vs_rvertex": ratio(self.found["rv"], self.denom["rv"]),
            "fake_rate_vs_pt": ratio(self.fake["pt"], self.cands["pt"]),
            "fake_rate_vs_eta": ratio(self.fake["eta"], self.cands["eta"]),
            "bins": {"pt": PT_BINS.tolist(), "eta": ETA_BINS.tolist(), "rvertex": RV_BINS.tolist()},
        }


def _events(geom, sample: str, n: int):
    if sample == "cube":
        return [synth.muon_cube_event(geom, 100 + i) for i in range(n)]
    return [synth.pileup_event(geom, 200 + i, pileup=200, mean_per_vertex=96, config=3) for i in range(n)]


def run_mode(ctx_factory, geom, cuts, flat, n_hidden, events) -> dict:
    """Track candidates of every event through the library with the given cut set."""
    ctx = ctx_factory()
    ctx.load_geometry(geom, cuts, flat, n_hidden)
    tally = Tally()
    n_t5 = 0
    from . import lst
    for e in events:
        ev = ctx.run_event(e.x, e.y, e.z, e.sensor)
        tc = ev.candidates(lst.LST_TC)[0]
        n_t5 += ev.counts()["t5"]
        ev.release()
        tally.add(tc, e, geom.layer)
    ctx.close()
    out = tally.result()
    out["t5_per_event"] = n_t5 / max(1, len(events))
    return out


def compare(sample="pu200", n_events=20, chi2_max=20.0, model="t5dnn_2x32.npz", precision="fp32",
            bisect_steps=12) -> dict:
    from . import lst, model_store
    w = model_store.load(f"{model_store.WEIGHTS_DIR}/{model}")
    geom = synth.build_geometry(True)
    events = _events(geom, sample, n_events)
    prec = {"fp32": lst.LST_FP32, "bf16": lst.LST_BF16, "bf16x3": lst.LST_BF16X3}[precision]
    factory = lambda: lst.Context(0, max_events=2, precision=prec)
    t0 = time.time()
    res = {"sample": sample, "events": n_events, "model": model, "precision": precision, "chi2_max": chi2_max}
    dnn = synth.open_cuts()
    dnn["wp"] = np.float32(w["wp"])
    res["dnn_trained_wp"] = dict(run_mode(factory, geom, dnn, w["flat"], w["n_hidden"], events), wp=float(w["wp"]))
    res["pre_dnn"] = run_mode(factory, geom, synth.pre_dnn_cuts(chi2_max), w["flat"], w["n_hidden"], events)
    target = res["pre_dnn"]["efficiency"]
    lo, hi = 0.0, 1.0                          # efficiency falls as the working point rises
    best = None
    for _ in range(bisect_steps):
        mid = 0.5 * (lo + hi)
        c = dict(dnn, wp=np.float32(mid))
        r = run_mode(factory, geom, c, w["flat"], w["n_hidden"], events)
        r["wp"] = mid
        if r["efficiency"] >= target:
            best, lo = r, mid
        else:
            hi = mid
    res["dnn_matched_wp"] = best
    res["seconds"] = round(time.time() - t0, 1)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sample", default="pu200", choices=["pu200", "cube"])
    ap.add_argument("--events", type=int, default=20)
    ap.add_argument("--chi2-max", type=float, default=20.0)
    ap.add_argument("--model", default="t5dnn_2x32.npz")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = compare(a.sample, a.events, a.chi2_max, a.model, a.precision)
    txt = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    for k in ("dnn_trained_wp", "pre_dnn", "dnn_matched_wp"):
        r = res[k] or {}
        print(f"{k:16s} eff {r.get('efficiency', math.nan):.4f}  fake {r.get('fake_rate', math.nan):.4f}  "
              f"dup {r.get('duplicate_rate', math.nan):.4f}  wp {r.get('wp', '-')}")


if __name__ == "__main__":
    main()
