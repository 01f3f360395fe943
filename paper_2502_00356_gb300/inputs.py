"""Seeded synthetic inputs for K_nu evaluation and Matern matrix generation.

This module holds no arithmetic of the method: it only draws inputs.  Both the
CUDA path and the oracle receive exactly these arrays.  All draws use numpy's
PCG64 generator (``np.random.default_rng(seed)``), which gives the same stream
on every platform.

Shapes follow the paper's workloads: locations in the unit square (Sec. V-D
rescales real data there), length scales in 0.02-0.3, smoothness 0.3-3.5
(Sec. V-C, Table I), and x = r / beta up to sqrt(2)/0.01 ~ 140 (Sec. IV-C).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def kv_pairs(n: int, seed: int, x_lo: float = 1e-3, x_hi: float = 140.0,
             nu_lo: float = 0.05, nu_hi: float = 10.0):
    """n pairs (x, nu): x log-uniform in [x_lo, x_hi], nu uniform in [nu_lo, nu_hi].

    x is drawn first, then nu, from one generator seeded with ``seed``.
    """
    rng = np.random.default_rng(seed)
    x = np.exp(rng.uniform(math.log(x_lo), math.log(x_hi), size=n))
    nu = rng.uniform(nu_lo, nu_hi, size=n)
    return np.ascontiguousarray(x), np.ascontiguousarray(nu)


def jittered_grid(n: int, seed: int, jitter: float = 0.4) -> np.ndarray:
    """n 2D locations on a jittered regular grid in the unit square.

    Grid side g = ceil(sqrt(n)), spacing s = 1/g.  Point k = i*g + j (row i,
    column j) sits at ((j + 1/2) s, (i + 1/2) s) + U(-jitter, jitter) * s per
    coordinate.  Points are kept in row-major order and truncated to the first
    n.  Returns the structure-of-arrays layout, shape (2, n):
    row 0 = x coordinates, row 1 = y coordinates.
    """
    if n < 0:
        raise ValueError("n must be >= 0")
    g = max(1, math.ceil(math.sqrt(n)))
    s = 1.0 / g
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter, jitter, size=(g * g, 2))
    ii, jj = np.divmod(np.arange(g * g), g)
    x = (jj + 0.5) * s + jit[:, 0] * s
    y = (ii + 0.5) * s + jit[:, 1] * s
    locs = np.stack([x, y])[:, :n]
    return np.ascontiguousarray(locs)


def morton_codes(locs: np.ndarray) -> np.ndarray:
    """Z-order codes of SoA locations in [0, 1]^2 (Sec. IV-D orders locations
    this way so that nearby distances share a block).

    Each coordinate is quantised to 16 bits, q = min(65535, floor(c * 65536))
    (clamped below at 0); x takes the even bits and y the odd bits of a 32-bit
    code.
    """
    locs = np.asarray(locs, dtype=np.float64)
    q = np.clip(np.floor(locs * 65536.0), 0, 65535).astype(np.uint64)
    code = np.zeros(locs.shape[1], dtype=np.uint64)
    for b in range(16):
        code |= ((q[0] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        code |= ((q[1] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return code


def morton_order(locs: np.ndarray) -> np.ndarray:
    """Permutation sorting locations by Morton code (stable: ties keep order)."""
    return np.argsort(morton_codes(locs), kind="stable").astype(np.int64)


def morton_sorted(locs: np.ndarray) -> np.ndarray:
    """Locations reordered by ``morton_order`` (SoA, contiguous)."""
    return np.ascontiguousarray(np.asarray(locs)[:, morton_order(locs)])


@dataclass
class MaternInstance:
    n: int
    seed: int
    sigma2: float
    beta: float
    nu: float

    def locations(self, morton: bool = True) -> np.ndarray:
        locs = jittered_grid(self.n, self.seed)
        return morton_sorted(locs) if morton else locs


def batched_instances(count: int = 256, seed: int = 99, n_lo: int = 500, n_hi: int = 8000,
                      sigma2_range=(0.5, 2.0), beta_range=(0.02, 0.3),
                      nu_range=(0.3, 3.0), first_instance_seed: int = 100):
    """A maximum-likelihood style parameter sweep: ``count`` Matern instances
    with n log-uniform in [n_lo, n_hi] and per-instance (sigma^2, beta, nu).
    Instance k draws its locations with seed first_instance_seed + k."""
    rng = np.random.default_rng(seed)
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)
    s2 = rng.uniform(*sigma2_range, size=count)
    be = rng.uniform(*beta_range, size=count)
    nu = rng.uniform(*nu_range, size=count)
    return [MaternInstance(int(ns[k]), first_instance_seed + k, float(s2[k]), float(be[k]),
                           float(nu[k])) for k in range(count)]


def entry_sample(n: int, m: int, seed: int, near_fraction: float = 0.01):
    """m (i, j) index pairs of an n x n matrix for sampled parity checks.

    Most pairs are uniform; a ``near_fraction`` share pairs i with a nearby
    index (|i - j| <= 3 in Morton order) to stress small distances.  Includes
    the corners and the diagonal element (0, 0).
    """
    rng = np.random.default_rng(seed)
    k_near = int(m * near_fraction)
    I = rng.integers(0, n, size=m)
    J = rng.integers(0, n, size=m)
    if k_near and n > 1:
        off = rng.integers(1, 4, size=k_near)
        J[:k_near] = np.clip(I[:k_near] - off, 0, n - 1)
    if m >= 4:
        I[-4:] = [0, n - 1, n - 1, 0]
        J[-4:] = [0, 0, n - 1, n - 1]
    return I.astype(np.int64), J.astype(np.int64)
