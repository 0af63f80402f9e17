"""Train the T5-DNN on the project's own synthetic events (the paper's Section 2 recipe on
synthetic data: quintuplets built by LST with the fit-quality selections opened up
(synth.open_cuts), labelled real when
more than 75% of their hits come from one particle, binary cross entropy, 2 hidden layers
of 32; 1, 3 and 4 hidden layers for comparison).

Features come from the library itself (lst_get_t5_features), i.e. exactly what the score
kernels see. The working point is the score at which the held-out real-T5 efficiency is
`--target-eff`. Writes model_store .npz files (flat FP32 weights, wp, metadata).

    python -m paper_2403_13166_gb300.train_t5dnn --events 30 --out-dir weights/
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import lst, model_store, synth, truth


def collect(n_events: int, first_index: int, config: int = 3):
    g = synth.build_geometry(True)
    cuts = synth.open_cuts()
    ctx = lst.Context(0, max_events=2)
    ctx.load_geometry(g, cuts, synth.mlp_flat(synth.xavier_mlp()), 2)
    feats, labels, ev_of = [], [], []
    for i in range(n_events):
        e = synth.pileup_event(g, first_index + i, pileup=200, mean_per_vertex=96, config=config)
        ev = ctx.run_event(e.x, e.y, e.z, e.sensor)
        hits, _, _ = ev.candidates(lst.LST_T5)
        f = ev.features()
        ev.release()
        feats.append(f)
        labels.append(truth.t5_labels(hits, e.pid))
        ev_of.append(np.full(len(f), i, np.int32))
    ctx.close()
    return np.concatenate(feats), np.concatenate(labels).astype(np.float32), np.concatenate(ev_of)


def train(X, y, n_hidden, epochs, seed, device):
    import torch
    torch.manual_seed(seed)
    layers, d = [], synth.N_FEATURES
    for _ in range(n_hidden):
        layers += [torch.nn.Linear(d, synth.HIDDEN), torch.nn.ReLU()]
        d = synth.HIDDEN
    layers.append(torch.nn.Linear(d, 1))
    net = torch.nn.Sequential(*layers).to(device)
    opt = torch.optim.Adam(net.parameters(), lr=2e-3)
    sched = torch.optim.lr_scheduler.CosineAnnealingLR(opt, T_max=epochs)
    Xt = torch.from_numpy(X).to(device)
    yt = torch.from_numpy(y).to(device)
    lossf = torch.nn.BCEWithLogitsLoss()
    n = len(Xt)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(n, device=device)
        tot = 0.0
        for b in range(0, n, 4096):
            idx = perm[b:b + 4096]
            opt.zero_grad()
            loss = lossf(net(Xt[idx]).squeeze(1), yt[idx])
            loss.backward()
            opt.step()
            tot += float(loss.detach()) * len(idx)
        sched.step()
        hist.append(tot / n)
    return net, hist


def flat_weights(net):
    Ws = [m.weight.detach().cpu().numpy().astype(np.float64) for m in net if hasattr(m, "weight")]
    bs = [m.bias.detach().cpu().numpy().astype(np.float64) for m in net if hasattr(m, "bias")]
    return synth.mlp_flat({"W": Ws, "b": bs})


def evaluate(net, X, y, device, target_eff):
    import torch
    with torch.no_grad():
        s = torch.sigmoid(net(torch.from_numpy(X).to(device)).squeeze(1)).cpu().numpy()
    real = y > 0.5
    wp = float(np.quantile(s[real], 1.0 - target_eff)) if real.any() else 0.5
    eff = float((s[real] >= wp).mean()) if real.any() else 0.0
    fake = float((s[~real] >= wp).mean()) if (~real).any() else 0.0
    order = np.argsort(-s)
    tp = np.cumsum(real[order]) / max(1, real.sum())
    fp = np.cumsum(~real[order]) / max(1, (~real).sum())
    auc = float(np.trapezoid(tp, fp)) if hasattr(np, "trapezoid") else float(np.trapz(tp, fp))
    return wp, eff, fake, auc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--events", type=int, default=30)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--target-eff", type=float, default=0.95)
    ap.add_argument("--out-dir", default=model_store.WEIGHTS_DIR)
    ap.add_argument("--depths", type=int, nargs="+", default=[2, 1, 3, 4])
    args = ap.parse_args()
    import torch
    device = torch.device("cuda:0")
    t0 = time.time()
    X, y, ev = collect(args.events, first_index=0)
    n_train_ev = int(round(0.8 * args.events))       # 80/20 split by event (Section 2)
    tr, te = ev < n_train_ev, ev >= n_train_ev
    summary = {"events": args.events, "t5": int(len(y)), "real_fraction": float(y.mean()),
               "collect_s": round(time.time() - t0, 1), "models": {}}
    os.makedirs(args.out_dir, exist_ok=True)
    for depth in args.depths:
        t1 = time.time()
        net, hist = train(X[tr], y[tr], depth, args.epochs, seed=2403 + depth, device=device)
        wp, eff, fake, auc = evaluate(net, X[te], y[te], device, args.target_eff)
        meta = {"hidden_layers": depth, "width": synth.HIDDEN, "loss": "binary cross entropy",
                "train_events": n_train_ev, "test_events": args.events - n_train_ev, "epochs": args.epochs,
                "final_train_loss": hist[-1], "test_auc": auc, "test_real_eff": eff, "test_fake_rate": fake,
                "target_eff": args.target_eff, "train_s": round(time.time() - t1, 1),
                "data": "synthetic PU200-like events, seeds 3000..3000+events-1",
                "cuts": "open_cuts (fit-quality tolerances of steps 3-4 opened)"}
        name = f"t5dnn_{depth}x32.npz"
        model_store.save(os.path.join(args.out_dir, name), flat_weights(net), depth, wp, meta)
        summary["models"][name] = {"wp": wp, **meta}
        print(json.dumps({"model": name, "wp": wp, "eff": eff, "fake": fake, "auc": auc}), flush=True)
    with open(os.path.join(args.out_dir, "training_summary.json"), "w") as f:
        json.dump(summary, f, indent=1)


if __name__ == "__main__":
    main()
