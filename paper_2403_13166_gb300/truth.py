"""Truth matching on synthetic events (validation and training labels, not timed).

Section 1 of the paper: a track candidate matches a simulated track when more than 75%
of its hits belong to that track. For a quintuplet (10 hits) that means at least 8.
"""
from __future__ import annotations

import numpy as np

MATCH_FRACTION = 0.75


def match_particle(hit_tuples: np.ndarray, pid: np.ndarray) -> np.ndarray:
    """For each row of original hit indices return the matched particle id or -1."""
    hit_tuples = np.asarray(hit_tuples)
    if hit_tuples.shape[0] == 0:
        return np.zeros(0, np.int64)
    p = pid[hit_tuples]                           # [n, k]
    n, k = p.shape
    need = int(np.floor(MATCH_FRACTION * k)) + 1  # strictly more than 75%
    best = np.full(n, -1, np.int64)
    for j in range(k):
        cand = p[:, j]
        cnt = (p == cand[:, None]).sum(1)
        ok = (cnt >= need) & (cand >= 0) & (best < 0)
        best = np.where(ok, cand, best)
    return best


def t5_labels(t5_hits: np.ndarray, pid: np.ndarray) -> np.ndarray:
    """1 for a real quintuplet (>= 8 of its 10 hits from one particle), else 0."""
    return (match_particle(t5_hits, pid) >= 0).astype(np.int8)


def efficiency(t5_hits: np.ndarray, pid: np.ndarray, denom_particles: np.ndarray) -> float:
    """Fraction of the given particles matched by at least one candidate."""
    m = match_particle(t5_hits, pid)
    found = np.isin(denom_particles, m[m >= 0])
    return float(found.mean()) if denom_particles.size else 1.0


def md_layers(sensor: np.ndarray, pid: np.ndarray, layer_of_module: np.ndarray, n_part: int):
    """Per particle, the set of layers holding a true mini-doublet: a lower and an upper
    hit of that particle in the same module."""
    out = [set() for _ in range(n_part)]
    ok = pid >= 0
    if not ok.any():
        return out
    key = np.unique(np.stack([pid[ok], sensor[ok] // 2, sensor[ok] % 2], 1), axis=0)
    seen = {}
    for p, m, s in key:
        seen.setdefault((int(p), int(m)), set()).add(int(s))
    for (p, m), ss in seen.items():
        if len(ss) == 2:
            out[p].add(int(layer_of_module[m]))
    return out


def _layer_chains(length: int = 5):
    """Every sequence of `length` layers linked by the module map's layer relation: barrel
    l -> l+1, any barrel layer -> first disk (7), disk d -> d+1 (one side per particle)."""
    nxt = {l: ([l + 1] if l <= 5 else []) + [7] for l in range(1, 7)}
    nxt.update({d: [d + 1] for d in range(7, 11)})
    nxt[11] = []
    out = []

    def walk(ch):
        if len(ch) == length:
            out.append(tuple(ch))
            return
        for n in nxt[ch[-1]]:
            walk(ch + [n])

    for start in range(1, 12):
        walk([start])
    return tuple(out)


T5_CHAINS = _layer_chains(5)


def findable_t5(sensor, pid, layer_of_module, n_part, chains=T5_CHAINS):
    """Particles with true mini-doublets in five layers that form a chain of the module map
    (five consecutive barrel layers, a barrel run continued into the disks, or five disks)."""
    lay = md_layers(sensor, pid, layer_of_module, n_part)
    return np.array([p for p in range(n_part) if any(set(c) <= lay[p] for c in chains)], np.int64)
