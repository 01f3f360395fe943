"""Write the training labels of the learned window (calls only the oracle).

Samples: x log-uniform in [1e-3, 140], nu uniform in [0.05, 20] (seed 7 by
default, drawn by paper_2502_00356_gb300.inputs.kv_pairs).  Labels: the
eps-window of Sec. IV-B for eps = 2^-23 (the FP32 form's window) by the
oracle's bracketing and bisection, and the smallest trapezoid interval count
within 1e-6 relative on that window.

    python oracle/make_window_labels.py [--n 2000000] [--seed 7] [--out PATH]

Output: an .npz with float32 labels (n x 4: t*, t0, t1, N), the generator's
seed, n and ranges, and the first 16 x and nu (float64) so that a reader can
regenerate the inputs with inputs.kv_pairs and check them.  Default path:
oracle/_build/window_labels_s{seed}_n{n}.npz.
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2502_00356_gb300 import inputs  # noqa: E402

LOG_EPS32 = -23.0 * math.log(2.0)
NODE_TOL = 1e-6


def default_path(n: int, seed: int) -> str:
    return os.path.join(HERE, "_build", f"window_labels_s{seed}_n{n}.npz")


def make(n: int, seed: int, out: str | None = None, chunk: int = 200_000) -> str:
    out = out or default_path(n, seed)
    os.makedirs(os.path.dirname(out), exist_ok=True)
    x, nu = inputs.kv_pairs(n, seed=seed, x_lo=1e-3, x_hi=140.0, nu_lo=0.05, nu_hi=20.0)
    labels = np.empty((n, 6), dtype=np.float64)
    for a in range(0, n, chunk):
        labels[a:a + chunk] = oracle.window_labels(x[a:a + chunk], nu[a:a + chunk], LOG_EPS32,
                                                   NODE_TOL)
    np.savez(out, labels=labels[:, [0, 1, 2, 4]].astype(np.float32), n=n, seed=seed,
             x_range=np.array([1e-3, 140.0]), nu_range=np.array([0.05, 20.0]),
             x_head=x[:16], nu_head=nu[:16], log_eps=LOG_EPS32, node_tol=NODE_TOL)
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    t0 = time.time()
    path = make(a.n, a.seed, a.out)
    print(f"{path} ({time.time() - t0:.1f} s)")
