"""Error map of the paper's refined algorithm (Algorithm 2) over its region,
the analogue of the paper's accuracy heatmaps (Sec. V-A) with the oracle in
place of the reference values it used: for each cell of an (x, nu) grid over
x in [0.1, 140] (the integral branch; below 0.1 Algorithm 2 takes Temme's
series, which converges to K) and nu in [0, 20], the largest relative error
of the fixed window [0, t1 = 9] with b bins against K_nu(x), for
b = 16, 40, 128.  Both sides are oracle functions (the GPU's fixed-window
form matches the oracle's to 2e-12, tests/test_gpu_paper_alg2.py).

    python oracle/alg2_error_map.py            # prints Markdown tables

Test infrastructure and documentation only, like the rest of oracle/.
"""
from __future__ import annotations

import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import oracle  # noqa: E402

X_EDGES = [0.1, 0.3, 1.0, 3.0, 10.0, 30.0, 70.0, 140.0]
NU_EDGES = [0.0, 1.0, 2.5, 5.0, 7.5, 10.0, 15.0, 20.0]
PER_CELL = 5  # sample points per axis inside a cell


def cell_points(lo, hi, log):
    if log:
        return np.exp(np.linspace(math.log(lo), math.log(hi), PER_CELL))
    return np.linspace(lo, hi, PER_CELL)


def error_map(bins: int) -> np.ndarray:
    m = np.zeros((len(NU_EDGES) - 1, len(X_EDGES) - 1))
    for i in range(len(NU_EDGES) - 1):
        nus = cell_points(NU_EDGES[i], NU_EDGES[i + 1], False)
        for j in range(len(X_EDGES) - 1):
            xs = cell_points(X_EDGES[j], X_EDGES[j + 1], True)
            X, V = (a.ravel() for a in np.meshgrid(xs, nus))
            _, ref = oracle.besselk(X, V, return_log=True)
            got = np.array([oracle.fixed_window_log_k(float(x), float(v), 9.0, bins)
                            for x, v in zip(X, V)])
            m[i, j] = float(np.max(np.abs(np.expm1(got - ref))))
    return m


def markdown(bins: int, m: np.ndarray) -> str:
    head = "| ν \\ x | " + " | ".join(f"{a:g}–{b:g}" for a, b in zip(X_EDGES, X_EDGES[1:])) + " |"
    rule = "|---|" + "---|" * (len(X_EDGES) - 1)
    rows = []
    for i in range(m.shape[0]):
        cells = " | ".join(f"{math.log10(max(v, 1e-17)):.1f}" for v in m[i])
        rows.append(f"| {NU_EDGES[i]:g}–{NU_EDGES[i + 1]:g} | {cells} |")
    return "\n".join([f"b = {bins}: log10 of the largest relative error per cell", "", head, rule] + rows)


def main() -> None:
    for b in (16, 40, 128):
        print(markdown(b, error_map(b)))
        print()


if __name__ == "__main__":
    main()
