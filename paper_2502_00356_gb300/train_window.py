"""Train the learned-window network on the GPU and save a checkpoint.

    python -m paper_2502_00356_gb300.train_window LABELS.npz OUT.bkw [--steps N] [--batch B]

LABELS.npz holds float32 labels (n x 4: t*, t0, t1, N) of the eps = 2^-23
window and the seed and ranges of their inputs, as written by the label
script beside the oracle (oracle/make_window_labels.py); the inputs (x, nu)
are regenerated here from the seeded generator and checked against the
stored first entries.  Training runs entirely in the
library's kernels (bk_learned_train: fused forward/backward per 128 samples,
Adam); this script only moves the arrays to the device and reports the loss.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def train(labels_path: str, out_path: str, steps: int = 60_000, batch: int = 8192,
          lr: float = 2e-3, seed: int = 1, init_seed: int = 0, report_every: int = 5000):
    import torch

    import paper_2502_00356_gb300 as bk

    from paper_2502_00356_gb300 import inputs

    bk.build()
    d = np.load(labels_path)
    n, s = int(d["n"]), int(d["seed"])
    xh, nh = inputs.kv_pairs(n, seed=s, x_lo=float(d["x_range"][0]), x_hi=float(d["x_range"][1]),
                             nu_lo=float(d["nu_range"][0]), nu_hi=float(d["nu_range"][1]))
    if not (np.array_equal(xh[:16], d["x_head"]) and np.array_equal(nh[:16], d["nu_head"])):
        raise ValueError("regenerated inputs do not match the label file")
    dev = torch.device("cuda")
    x = torch.as_tensor(xh, device=dev)
    nu = torch.as_tensor(nh, device=dev)
    l4 = torch.as_tensor(d["labels"], device=dev).double()
    lab = torch.zeros((n, 6), dtype=torch.float64, device=dev)
    lab[:, 0:3] = l4[:, 0:3]
    lab[:, 4] = l4[:, 3]
    model = bk.LearnedWindow(seed=init_seed)
    loss = torch.zeros(steps, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    model.train(x, nu, lab, steps=steps, batch=batch, lr=lr, seed=seed, loss=loss)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    model.save(out_path)
    curve = loss.cpu().numpy()
    summary = {
        "labels": labels_path.split("/")[-1], "samples": int(x.numel()), "steps": steps,
        "batch": batch, "lr": lr, "seed": seed, "init_seed": init_seed, "train_seconds": dt,
        "loss_first": float(curve[:100].mean()), "loss_last": float(curve[-1000:].mean()),
        "loss_every": {str(k): float(curve[max(0, k - 100):k + 1].mean())
                       for k in range(0, steps, report_every)},
        "target_stats": [float(v) for v in model.stats()],
    }
    return model, summary


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("labels")
    ap.add_argument("out")
    ap.add_argument("--steps", type=int, default=60_000)
    ap.add_argument("--batch", type=int, default=8192)
    ap.add_argument("--lr", type=float, default=2e-3)
    a = ap.parse_args()
    _, s = train(a.labels, a.out, steps=a.steps, batch=a.batch, lr=a.lr)
    print(json.dumps(s))
