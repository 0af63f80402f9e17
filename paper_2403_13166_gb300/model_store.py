"""T5-DNN weight files: little-endian float32 network weights plus the working point.

Layout of the .npz written by the training tool: `flat` (float32, the lst_mlp flat layout
W0, b0, [Wh, bh]*, Wout, bout), `n_hidden` (int), `wp` (float32 working point), `meta`
(JSON text: training events, epochs, loss, efficiency at the working point)."""
from __future__ import annotations

import json
import os

import numpy as np

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
DEFAULT = os.path.join(WEIGHTS_DIR, "t5dnn_2x32.npz")


def save(path: str, flat: np.ndarray, n_hidden: int, wp: float, meta: dict) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, flat=np.asarray(flat, "<f4"), n_hidden=np.int32(n_hidden), wp=np.float32(wp),
             meta=np.array(json.dumps(meta)))


def load(path: str) -> dict:
    z = np.load(path)
    return {"flat": z["flat"].astype(np.float64), "n_hidden": int(z["n_hidden"]), "wp": float(z["wp"]),
            "meta": json.loads(str(z["meta"]))}


def load_trained(path: str = DEFAULT):
    """The project-trained 2x32 network if present, else None."""
    return load(path) if os.path.exists(path) else None
