"""CPU oracle for the K_nu / Matern hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.  ``oracle.cpp`` holds the arithmetic (long double);
this module builds it with the host C++ compiler and wraps it with ctypes.

Functions and the passages they follow:

* ``log_besselk`` / ``besselk``: K_nu(x) by the integral of Eq. (integral),
  Sec. IV-B, dense trapezoid with halving.
* ``besselk_temme``: Temme's series + Campbell's recurrence, Sec. IV-A
  (independent cross-check for small x).
* ``window``: the epsilon-window [t0, t1] around t_max, Sec. IV-B.
* ``min_nodes``: smallest trapezoid interval count on that window meeting a
  relative tolerance.
* ``matern_entries`` / ``matern_block``: the Matern covariance of Sec. III-A
  with sigma^2 where r == 0 (Algorithm 3).
* ``fixed_window_log_k``: the paper's fixed-window branch of Algorithm 2.
* ``besselk_f64`` / ``matern_entries_f64``: the same dense trapezoid in FP64
  (one template with the long double version), for samples of 10^5..10^6
  points where software binary128 (aarch64) would take minutes.
* ``mlp_*``: FP64 reference forward/backward of the window network (see
  ``mlp.py``).

``alg2_error_map.py`` (a script beside this package) tabulates the error of
the paper's Algorithm 2 over its region from these functions alone.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

LOG_EPS64 = -52.0 * np.log(2.0)  # log(2^-52), the paper's machine epsilon (Sec. IV-C)


def build(force: bool = False) -> str:
    """Compile oracle.cpp into _build/liboracle.so with g++ and OpenMP."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fopenmp",
           "-fno-fast-math", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        D, I64, I, P = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        sig = {
            "oracle_long_double_digits": (I, []),
            "oracle_max_threads": (I, []),
            "oracle_log_besselk": (D, [D, D, P]),
            "oracle_besselk": (D, [D, D]),
            "oracle_besselk_batch": (None, [P, P, P, P, I64, I]),
            "oracle_besselk_temme": (D, [D, D, P]),
            "oracle_besselk_grad_batch": (None, [P, P, P, P, P, I64, I]),
            "oracle_window": (None, [D, D, D, P]),
            "oracle_window_batch": (None, [P, P, D, P, I64, I]),
            "oracle_window_trapezoid_log_k": (D, [D, D, D, D, I64]),
            "oracle_min_nodes": (I64, [D, D, D, D, I64]),
            "oracle_min_nodes_batch": (None, [P, P, D, D, I64, P, I64, I]),
            "oracle_window_labels_batch": (None, [P, P, D, D, I64, P, I64, I]),
            "oracle_fixed_window_log_k": (D, [D, D, D, I64]),
            "oracle_matern_entries": (None, [P, I64, P, P, I64, D, D, D, P, I]),
            "oracle_matern_block": (None, [P, I64, P, I64, D, D, D, P, I64, I]),
            "oracle_besselk_batch_f64": (None, [P, P, P, P, I64, I]),
            "oracle_matern_entries_f64": (None, [P, I64, P, P, I64, D, D, D, P, I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _bcast(x, nu):
    """Broadcast x and nu; return (shape, flat x, flat nu) as contiguous float64."""
    x = np.asarray(x, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    shape = np.broadcast_shapes(x.shape, nu.shape)
    xa = np.ascontiguousarray(np.broadcast_to(x, shape).reshape(-1))
    na = np.ascontiguousarray(np.broadcast_to(nu, shape).reshape(-1))
    return shape, xa, na


def long_double_mantissa_bits() -> int:
    return _load().oracle_long_double_digits()


def max_threads() -> int:
    return _load().oracle_max_threads()


def log_besselk(x: float, nu: float) -> float:
    st = ctypes.c_int(0)
    v = _load().oracle_log_besselk(float(x), float(nu), ctypes.byref(st))
    return v if st.value == 0 else float("nan")


def besselk(x, nu, threads: int = 0, return_log: bool = False):
    """K_nu(x), elementwise over broadcast arrays (OpenMP over elements)."""
    shape, xa, na = _bcast(x, nu)
    out = np.empty_like(xa)
    lout = np.empty_like(xa)
    _load().oracle_besselk_batch(_ptr(xa), _ptr(na), _ptr(out), _ptr(lout), xa.size, int(threads))
    if return_log:
        return out.reshape(shape)[()], lout.reshape(shape)[()]
    return out.reshape(shape)[()]


def besselk_f64(x, nu, threads: int = 0, return_log: bool = False):
    """K_nu(x) by the FP64 instance of the dense trapezoid (OpenMP)."""
    shape, xa, na = _bcast(x, nu)
    out = np.empty_like(xa)
    lout = np.empty_like(xa)
    _load().oracle_besselk_batch_f64(_ptr(xa), _ptr(na), _ptr(out), _ptr(lout), xa.size,
                                     int(threads))
    if return_log:
        return out.reshape(shape)[()], lout.reshape(shape)[()]
    return out.reshape(shape)[()]


def besselk_grad(x, nu, threads: int = 0):
    """(K_nu(x), dK/dx, dK/dnu) elementwise over broadcast arrays, the
    derivatives by the integral differentiated under the sign."""
    shape, xf, nf = _bcast(x, nu)
    k, dx, dn = (np.empty(xf.size) for _ in range(3))
    _load().oracle_besselk_grad_batch(_ptr(xf), _ptr(nf), _ptr(k), _ptr(dx), _ptr(dn), xf.size,
                                      int(threads))
    return k.reshape(shape), dx.reshape(shape), dn.reshape(shape)


def besselk_temme(x: float, nu: float) -> float:
    st = ctypes.c_int(0)
    v = _load().oracle_besselk_temme(float(x), float(nu), ctypes.byref(st))
    return v if st.value == 0 else float("nan")


def window(x, nu, log_eps: float = LOG_EPS64, threads: int = 0) -> np.ndarray:
    """Rows (t*, t0, t1, g(t*)) for each (x, nu)."""
    _, xa, na = _bcast(x, nu)
    out = np.empty((xa.size, 4), dtype=np.float64)
    _load().oracle_window_batch(_ptr(xa), _ptr(na), float(log_eps), _ptr(out), xa.size, int(threads))
    return out


def window_trapezoid_log_k(x: float, nu: float, t0: float, t1: float, n_intervals: int) -> float:
    return _load().oracle_window_trapezoid_log_k(float(x), float(nu), float(t0), float(t1),
                                                 int(n_intervals))


def min_nodes(x, nu, rel_tol: float, log_eps: float = LOG_EPS64, nmax: int = 512,
              threads: int = 0) -> np.ndarray:
    _, xa, na = _bcast(x, nu)
    out = np.empty(xa.size, dtype=np.int64)
    _load().oracle_min_nodes_batch(_ptr(xa), _ptr(na), float(log_eps), float(rel_tol), int(nmax),
                                   _ptr(out), xa.size, int(threads))
    return out


def window_labels(x, nu, log_eps: float, rel_tol: float, nmax: int = 256,
                  threads: int = 0) -> np.ndarray:
    """Rows (t*, t0, t1, g(t*), N, log T_ref) of the eps-window labels."""
    _, xa, na = _bcast(x, nu)
    out = np.empty((xa.size, 6), dtype=np.float64)
    _load().oracle_window_labels_batch(_ptr(xa), _ptr(na), float(log_eps), float(rel_tol),
                                       int(nmax), _ptr(out), xa.size, int(threads))
    return out


def fixed_window_log_k(x: float, nu: float, t1: float = 9.0, bins: int = 40) -> float:
    return _load().oracle_fixed_window_log_k(float(x), float(nu), float(t1), int(bins))


def matern_entries(locs: np.ndarray, I, J, sigma2: float, beta: float, nu: float,
                   threads: int = 0) -> np.ndarray:
    """Entries M[I[k], J[k]] for SoA locations of shape (2, n)."""
    locs = _f64(locs)
    assert locs.ndim == 2 and locs.shape[0] == 2
    n = locs.shape[1]
    I = np.ascontiguousarray(np.asarray(I, dtype=np.int64))
    J = np.ascontiguousarray(np.asarray(J, dtype=np.int64))
    assert I.shape == J.shape
    if I.size and (I.min() < 0 or J.min() < 0 or I.max() >= n or J.max() >= n):
        raise IndexError("entry index out of range")
    out = np.empty(I.size, dtype=np.float64)
    _load().oracle_matern_entries(_ptr(locs), n, _ptr(I), _ptr(J), I.size, float(sigma2),
                                  float(beta), float(nu), _ptr(out), int(threads))
    return out


def matern_entries_f64(locs: np.ndarray, I, J, sigma2: float, beta: float, nu: float,
                       threads: int = 0) -> np.ndarray:
    """Entries M[I[k], J[k]] by the FP64 instance of the oracle."""
    locs = _f64(locs)
    assert locs.ndim == 2 and locs.shape[0] == 2
    n = locs.shape[1]
    I = np.ascontiguousarray(np.asarray(I, dtype=np.int64))
    J = np.ascontiguousarray(np.asarray(J, dtype=np.int64))
    assert I.shape == J.shape
    if I.size and (I.min() < 0 or J.min() < 0 or I.max() >= n or J.max() >= n):
        raise IndexError("entry index out of range")
    out = np.empty(I.size, dtype=np.float64)
    _load().oracle_matern_entries_f64(_ptr(locs), n, _ptr(I), _ptr(J), I.size, float(sigma2),
                                      float(beta), float(nu), _ptr(out), int(threads))
    return out


def matern_block(locs1: np.ndarray, locs2: np.ndarray, sigma2: float, beta: float, nu: float,
                 threads: int = 0) -> np.ndarray:
    """Dense m x n block (returned as a numpy array indexed [i, j])."""
    l1, l2 = _f64(locs1), _f64(locs2)
    m, n = l1.shape[1], l2.shape[1]
    out = np.empty((n, m), dtype=np.float64)  # column-major m x n == row-major n x m
    _load().oracle_matern_block(_ptr(l1), m, _ptr(l2), n, float(sigma2), float(beta), float(nu),
                                _ptr(out), m, int(threads))
    return out.T.copy()
