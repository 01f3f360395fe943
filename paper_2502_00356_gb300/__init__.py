"""Python binding of libbesselk (include/bk.h): K_nu(x) and Matern covariance
matrices on one GB300.

The functions here have the C-ABI's names and only marshal arguments: they
check tensor devices, dtypes and shapes, pass raw device pointers and the
current torch CUDA stream, and raise ``BkError`` on a non-OK status.  Every
step of the computation runs in the library's CUDA kernels; there is no CPU
fallback, and calling any of them without the built library raises.

PyTorch provides device memory and streams only.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

from . import inputs  # noqa: F401  (seeded generators; no method arithmetic)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbesselk.so")

BK_OK, BK_ERR_INVALID_ARG, BK_ERR_CUDA, BK_ERR_NOMEM = 0, 1, 2, 3
BK_ERR_UNSUPPORTED, BK_ERR_NOT_CONVERGED, BK_ERR_NOT_LOADED = 4, 5, 6
BK_F64, BK_F32 = 0, 1
BK_WIN_SEARCH, BK_WIN_LEARNED, BK_WIN_FIXED = 0, 1, 2
BK_CTR_FALLBACK, BK_CTR_FAIL, BK_CTR_NODES, BK_CTR_ITERS, BK_CTR_EVALS, BK_CTR_PEAK_ITERS = 0, 1, 2, 3, 4, 5
BK_CTR_REPAIR, BK_CTR_SERIES = 6, 7
BK_NUM_COUNTERS = 8
BK_HOST_AUTO, BK_HOST_STAGED = 0, 1
BK_TRAIN_TENSOR, BK_TRAIN_SIMT = 0, 1

#: every symbol include/bk.h declares (checked by the CPU tests)
EXPORTS = (
    "bk_opts_default", "bk_version", "bk_last_error", "bk_status_string", "bk_sync",
    "bk_eval", "bk_eval_ex", "bk_eval_grad", "bk_eval_autotune", "bk_gaussian_loglik", "bk_matern_tile", "bk_matern_tile_ex", "bk_matern_tile2",
    "bk_matern_tile_host", "bk_matern_tile_host_workspace",
    "bk_morton_order", "bk_probe_pipe", "bk_math_probe", "bk_batched_plan_create", "bk_batched_plan_destroy",
    "bk_batched_plan_info", "bk_batched_autotune", "bk_matern_batched",
    "bk_matern_batched_static", "bk_learned_create", "bk_learned_destroy", "bk_learned_train",
    "bk_learned_grad", "bk_learned_infer", "bk_learned_params", "bk_learned_stats",
    "bk_learned_set_margins", "bk_learned_set_train_path", "bk_learned_save", "bk_learned_load",
)


class BkError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_STATUS = {0: "BK_OK", 1: "BK_ERR_INVALID_ARG", 2: "BK_ERR_CUDA", 3: "BK_ERR_NOMEM",
           4: "BK_ERR_UNSUPPORTED", 5: "BK_ERR_NOT_CONVERGED", 6: "BK_ERR_NOT_LOADED"}


class bk_opts(ctypes.Structure):
    _fields_ = [("window", ctypes.c_int), ("compute", ctypes.c_int), ("fixed_bins", ctypes.c_int),
                ("fixed_t1", ctypes.c_double), ("d_counters", ctypes.c_void_p),
                ("learned", ctypes.c_void_p), ("search_f64", ctypes.c_int),
                ("series_below", ctypes.c_double), ("d_cosh_table", ctypes.c_void_p),
                ("lanes", ctypes.c_int)]


_lock = threading.Lock()
_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA library (nvcc, sm_103a) into the package's _build/."""
    from .buildlib import build as _build
    return _build(force=force, verbose=verbose)


def lib() -> ctypes.CDLL:
    """Load libbesselk.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libbesselk is not built ({LIB_PATH} missing); "
                               "run paper_2502_00356_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        sig = {
            "bk_opts_default": (None, [P]),
            "bk_version": (ctypes.c_char_p, []),
            "bk_last_error": (ctypes.c_char_p, []),
            "bk_status_string": (ctypes.c_char_p, [I]),
            "bk_sync": (I, [P]),
            "bk_eval": (I, [P, P, P, I64, P]),
            "bk_eval_ex": (I, [P, P, P, P, I, I64, P, P]),
            "bk_eval_grad": (I, [P, P, P, P, P, I64, P, P]),
            "bk_eval_autotune": (I, [P, P, P, I, I64, P, P, P]),
            "bk_gaussian_loglik": (I, [P, I64, I64, P, P, P, P, P]),
            "bk_matern_tile": (I, [P, I64, D, D, D, P, I64, I, P]),
            "bk_matern_tile_ex": (I, [P, I64, D, D, D, P, I64, I, P, P]),
            "bk_matern_tile2": (I, [P, I64, P, I64, D, D, D, P, I64, I, P, P]),
            "bk_matern_tile_host": (I, [P, I64, D, D, D, P, I64, I, P, I, P, ctypes.c_size_t, P]),
            "bk_matern_tile_host_workspace": (ctypes.c_size_t, [I64, I, I]),
            "bk_morton_order": (I, [P, I64, P]),
            "bk_probe_pipe": (I, [I, I64, I, I, P, P]),
            "bk_math_probe": (I, [I, P, P, I64, P]),
            "bk_batched_plan_create": (I, [P, P, ctypes.c_int32, I, P]),
            "bk_batched_plan_destroy": (I, [P]),
            "bk_batched_plan_info": (I, [P, P, P, P, P, P]),
            "bk_batched_autotune": (I, [P, P, I64, P]),
            "bk_matern_batched": (I, [P, ctypes.c_int32, I, P, P]),
            "bk_matern_batched_static": (I, [P, ctypes.c_int32, I, P]),
            "bk_learned_create": (I, [P, ctypes.c_uint64]),
            "bk_learned_destroy": (I, [P]),
            "bk_learned_train": (I, [P, P, P, P, I64, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_float, ctypes.c_uint64, P, P]),
            "bk_learned_grad": (I, [P, P, P, P, I64, P, P, P]),
            "bk_learned_infer": (I, [P, P, P, P, I64, P]),
            "bk_learned_params": (I, [P, P, P]),
            "bk_learned_stats": (I, [P, P, P]),
            "bk_learned_set_margins": (I, [P, ctypes.c_float, ctypes.c_float]),
            "bk_learned_set_train_path": (I, [P, ctypes.c_int]),
            "bk_learned_save": (I, [P, ctypes.c_char_p]),
            "bk_learned_load": (I, [P, ctypes.c_char_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _check(status: int) -> None:
    if status != BK_OK:
        msg = lib().bk_last_error().decode(errors="replace")
        raise BkError(status, msg)


def last_error() -> str:
    return lib().bk_last_error().decode(errors="replace")


def version() -> str:
    return lib().bk_version().decode()


# ---------------------------------------------------------------------------
# torch marshalling helpers
def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> Optional[int]:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _dev(t, name: str, dtype=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t) -> Optional[int]:
    return None if t is None else (t.data_ptr() or None)


def make_opts(window: int = BK_WIN_SEARCH, compute: int = BK_F64, fixed_bins: int = 40,
              fixed_t1: float = 9.0, counters=None, learned=None,
              search_f64: bool = False, series_below: float = 0.0, lanes: int = 0) -> bk_opts:
    """A bk_opts struct; ``counters`` is an optional CUDA int64 tensor of
    BK_NUM_COUNTERS entries that kernels add to; ``learned`` a LearnedWindow
    (implies window = BK_WIN_LEARNED and compute = BK_F32 unless given);
    ``search_f64`` makes the plain form run the FP64 Newton search for every
    point instead of taking FP32 roots checked in FP64; ``series_below`` is the
    x below which the plain form uses Temme's series (0: never).  The paper's
    refined algorithm (Algorithm 2) is ``paper_algorithm2_opts()``."""
    o = bk_opts()
    lib().bk_opts_default(ctypes.byref(o))
    if learned is not None:
        if window == BK_WIN_SEARCH:
            window = BK_WIN_LEARNED
        if compute == BK_F64:
            compute = BK_F32
        o.learned = learned.handle.value
    o.window, o.compute, o.fixed_bins, o.fixed_t1 = int(window), int(compute), int(fixed_bins), float(fixed_t1)
    o.search_f64 = int(bool(search_f64))
    o.series_below = float(series_below)
    o.lanes = int(lanes)
    if counters is not None:
        torch = _torch()
        _dev(counters, "counters", torch.int64)
        if counters.numel() < BK_NUM_COUNTERS:
            raise ValueError("counters needs BK_NUM_COUNTERS entries")
        o.d_counters = counters.data_ptr()
    return o



def paper_algorithm2_opts(bins: int = 40, t1: float = 9.0, series_below: float = 0.1,
                          counters=None) -> bk_opts:
    """Options for the paper's refined algorithm (Algorithm 2): Temme's series
    below x = 0.1, else the fixed window [0, 9] with 40 bins (plain FP64)."""
    return make_opts(window=BK_WIN_FIXED, fixed_bins=bins, fixed_t1=t1,
                     series_below=series_below, counters=counters)

def _dtype_code(torch_dtype) -> int:
    torch = _torch()
    if torch_dtype == torch.float64:
        return BK_F64
    if torch_dtype == torch.float32:
        return BK_F32
    raise TypeError("output dtype must be float64 or float32")


def _torch_dtype(code: int):
    torch = _torch()
    return {BK_F64: torch.float64, BK_F32: torch.float32}[code]


# ---------------------------------------------------------------------------
# entry points (same names as the C-ABI)
def bk_eval(x, nu, out=None, stream=None):
    """out = K_nu(x), FP64 plain form.  x, nu: CUDA float64 tensors of equal size."""
    torch = _torch()
    _dev(x, "x", torch.float64)
    _dev(nu, "nu", torch.float64)
    if x.numel() != nu.numel():
        raise ValueError("x and nu must have the same number of elements")
    if out is None:
        out = torch.empty_like(x)
    _dev(out, "out", torch.float64)
    if out.numel() != x.numel():
        raise ValueError("out has the wrong size")
    _check(lib().bk_eval(_ptr(x), _ptr(nu), _ptr(out), x.numel(), _stream_ptr(stream)))
    return out


def bk_eval_ex(x, nu, out=None, log_out=None, out_dtype=None, opts: Optional[bk_opts] = None,
               stream=None, want_log: bool = False):
    """K_nu(x) (and optionally log K_nu(x)) with options; returns (out, log_out)."""
    torch = _torch()
    _dev(x, "x", torch.float64)
    _dev(nu, "nu", torch.float64)
    n = x.numel()
    if nu.numel() != n:
        raise ValueError("x and nu must have the same number of elements")
    if out_dtype is None:
        out_dtype = out.dtype if out is not None else torch.float64
    code = _dtype_code(out_dtype)
    if out is None:
        out = torch.empty(x.shape, dtype=out_dtype, device=x.device)
    _dev(out, "out", out_dtype)
    if want_log and log_out is None:
        log_out = torch.empty(x.shape, dtype=out_dtype, device=x.device)
    if log_out is not None:
        _dev(log_out, "log_out", out_dtype)
    optp = ctypes.byref(opts) if opts is not None else None
    _check(lib().bk_eval_ex(_ptr(x), _ptr(nu), _ptr(out), _ptr(log_out), code, n, optp,
                            _stream_ptr(stream)))
    return out, log_out


def bk_eval_autotune(x, nu, out, opts: bk_opts, stream=None) -> int:
    """Times the FP32 forms' bare evaluation with 1, 2, 4 and 8 lanes per
    evaluation on (up to 2^20 of) these pairs, keeps the fastest for later
    calls with lanes = 0 in this process and returns it (synchronises)."""
    torch = _torch()
    _dev(x, "x", torch.float64)
    _dev(nu, "nu", torch.float64)
    _dev(out, "out")
    if nu.numel() != x.numel() or out.numel() != x.numel():
        raise ValueError("x, nu and out must have the same number of elements")
    best = ctypes.c_int(0)
    _check(lib().bk_eval_autotune(_ptr(x), _ptr(nu), _ptr(out), _dtype_code(out.dtype), x.numel(),
                                  ctypes.byref(opts), _stream_ptr(stream), ctypes.byref(best)))
    return best.value


def bk_eval_grad(x, nu, k=None, dk_dx=None, dk_dnu=None, opts: Optional[bk_opts] = None,
                 stream=None):
    """(K_nu(x), dK/dx, dK/dnu) of the plain FP64 form from one quadrature;
    x, nu: CUDA float64 tensors of equal size.  Returns the three tensors."""
    torch = _torch()
    _dev(x, "x", torch.float64)
    _dev(nu, "nu", torch.float64)
    n = x.numel()
    if nu.numel() != n:
        raise ValueError("x and nu must have the same number of elements")
    outs = []
    for t, name in ((k, "k"), (dk_dx, "dk_dx"), (dk_dnu, "dk_dnu")):
        if t is None:
            t = torch.empty(x.shape, dtype=torch.float64, device=x.device)
        _dev(t, name, torch.float64)
        if t.numel() != n:
            raise ValueError(f"{name} has the wrong size")
        outs.append(t)
    optp = ctypes.byref(opts) if opts is not None else None
    _check(lib().bk_eval_grad(_ptr(x), _ptr(nu), _ptr(outs[0]), _ptr(outs[1]), _ptr(outs[2]), n,
                              optp, _stream_ptr(stream)))
    return tuple(outs)


def bk_gaussian_loglik(a, z, y=None, out=None, opts: Optional[bk_opts] = None, stream=None):
    """Gaussian log-likelihood of z under the covariance ``a`` (CUDA float64,
    viewed column-major like the Matern outputs: shape (n, ld), its lower
    triangle overwritten by the Cholesky factor).  Returns ``out`` =
    [l, log det a, z^T a^{-1} z] (CUDA float64, 3)."""
    torch = _torch()
    _dev(a, "a", torch.float64)
    _dev(z, "z", torch.float64)
    if a.dim() != 2:
        raise ValueError("a must be 2-D (n, ld)")
    n, ld = a.shape[0], a.shape[1]
    if z.numel() != n:
        raise ValueError("z must have n elements")
    if y is None:
        y = torch.empty(n, dtype=torch.float64, device=a.device)
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=a.device)
    _dev(y, "y", torch.float64)
    _dev(out, "out", torch.float64)
    optp = ctypes.byref(opts) if opts is not None else None
    _check(lib().bk_gaussian_loglik(_ptr(a), n, ld, _ptr(z), _ptr(y), _ptr(out), optp,
                                    _stream_ptr(stream)))
    return out


def _locs(locs, name="locs"):
    torch = _torch()
    _dev(locs, name, torch.float64)
    if locs.dim() != 2 or locs.shape[0] != 2:
        raise ValueError(f"{name} must have shape (2, n) (structure of arrays)")
    return locs.shape[1]


BK_COSH_TABLE_LEN = 3328


def _with_cosh_table(opts, device, dtype_code):
    """A copy of ``opts`` whose d_cosh_table is a scratch tensor from torch's
    caching allocator on the current stream (so the library allocates nothing
    and graph capture takes it from the graph's pool); returns (opts, tensor
    keeping the scratch alive).  ``opts`` None means the C defaults for a
    NULL options pointer: default options with compute = the output dtype
    (FP32 output takes the FP32 precision form)."""
    torch = _torch()
    if opts is None:
        o = bk_opts()
        lib().bk_opts_default(ctypes.byref(o))
        o.compute = int(dtype_code)
    else:
        o = bk_opts.from_buffer_copy(opts)
    table = None
    if not o.d_cosh_table:
        table = torch.empty(BK_COSH_TABLE_LEN, dtype=torch.float64, device=device)
        o.d_cosh_table = table.data_ptr()
    return o, table


def bk_matern_tile(locs, sigma2: float, beta: float, nu: float, out=None, dtype=None,
                   opts: Optional[bk_opts] = None, stream=None):
    """Full n x n Matern matrix of SoA locations (2, n).  ``out`` is a CUDA
    tensor viewed column-major: out[j, i] holds entry (i, j), i.e. pass a
    (n, ld) row-major tensor; returns it."""
    torch = _torch()
    n = _locs(locs)
    if out is None:
        out = torch.empty((n, n), dtype=dtype or torch.float64, device=locs.device)
    code = _dtype_code(out.dtype)
    _dev(out, "out")
    if out.dim() != 2 or out.shape[0] != n or out.shape[1] < n:
        raise ValueError("out must be (n, ld) with ld >= n")
    ld = out.shape[1]
    o, table = _with_cosh_table(opts, locs.device, code)
    _check(lib().bk_matern_tile_ex(_ptr(locs), n, float(sigma2), float(beta), float(nu), _ptr(out),
                                   ld, code, ctypes.byref(o), _stream_ptr(stream)))
    del table  # stream-ordered reuse by torch's allocator is safe after the launch
    return out


def matern_tile_host_workspace(n: int, dtype=None, staged: bool = True) -> int:
    """Bytes of device workspace bk_matern_tile_host needs for n locations:
    staged=True for pageable output (the matrix passes through the
    workspace), False for page-locked output (written directly)."""
    torch = _torch()
    return int(lib().bk_matern_tile_host_workspace(int(n), _dtype_code(dtype or torch.float64),
                                                   int(bool(staged))))


def bk_matern_tile_host(locs, sigma2: float, beta: float, nu: float, out, work,
                        opts: Optional[bk_opts] = None, staged: bool = False, stream=None):
    """The n x n Matern matrix of HOST locations ``locs`` (a (2, n) float64 CPU
    tensor) written into the HOST tensor ``out`` ((n, ld) row-major =
    column-major n x n, float64 or float32), with ``work`` a CUDA uint8 tensor
    of at least matern_tile_host_workspace(n, staged=...) bytes.  By default
    the kernel stores into ``out`` directly when the device can address it;
    ``staged=True`` generates the matrix in ``work`` and copies finished
    panels out.  Asynchronous on ``stream``: ``out`` is complete once the
    stream has reached the end of the call.  Returns ``out``."""
    torch = _torch()
    if not isinstance(locs, torch.Tensor) or locs.is_cuda or locs.dtype != torch.float64:
        raise TypeError("locs must be a float64 CPU tensor")
    if locs.dim() != 2 or locs.shape[0] != 2 or not locs.is_contiguous():
        raise ValueError("locs must be a contiguous (2, n) tensor (structure of arrays)")
    n = locs.shape[1]
    if not isinstance(out, torch.Tensor) or out.is_cuda or not out.is_contiguous():
        raise TypeError("out must be a contiguous CPU tensor")
    if out.dim() != 2 or out.shape[0] != n or out.shape[1] < n:
        raise ValueError("out must be (n, ld) with ld >= n")
    code = _dtype_code(out.dtype)
    _dev(work, "work")
    o = opts
    if o is None:
        o = bk_opts()
        lib().bk_opts_default(ctypes.byref(o))
        o.compute = code
    _check(lib().bk_matern_tile_host(_ptr(locs), n, float(sigma2), float(beta), float(nu),
                                     _ptr(out), out.shape[1], code, ctypes.byref(o),
                                     BK_HOST_STAGED if staged else BK_HOST_AUTO, _ptr(work),
                                     work.numel() * work.element_size(), _stream_ptr(stream)))
    return out


def bk_matern_tile2(locs1, locs2, sigma2: float, beta: float, nu: float, out=None, dtype=None,
                    opts: Optional[bk_opts] = None, stream=None):
    """m x n block between locs1 (2, m) and locs2 (2, n); ``out`` is (n, ld)
    row-major = column-major m x n with leading dimension ld >= m."""
    torch = _torch()
    m = _locs(locs1, "locs1")
    n = _locs(locs2, "locs2")
    if out is None:
        out = torch.empty((n, m), dtype=dtype or torch.float64, device=locs1.device)
    code = _dtype_code(out.dtype)
    _dev(out, "out")
    if out.dim() != 2 or out.shape[0] != n or out.shape[1] < m:
        raise ValueError("out must be (n, ld) with ld >= m")
    o, table = _with_cosh_table(opts, locs1.device, code)
    _check(lib().bk_matern_tile2(_ptr(locs1), m, _ptr(locs2), n, float(sigma2), float(beta),
                                 float(nu), _ptr(out), out.shape[1], code, ctypes.byref(o),
                                 _stream_ptr(stream)))
    return out


def bk_morton_order(locs_host) -> "object":
    """Host-side Z-order permutation of SoA locations (numpy array (2, n))."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(locs_host, dtype=np.float64))
    if a.ndim != 2 or a.shape[0] != 2:
        raise ValueError("locs must have shape (2, n)")
    perm = np.empty(a.shape[1], dtype=np.int64)
    _check(lib().bk_morton_order(a.ctypes.data_as(ctypes.c_void_p), a.shape[1],
                                 perm.ctypes.data_as(ctypes.c_void_p)))
    return perm


def bk_sync(stream=None):
    _check(lib().bk_sync(_stream_ptr(stream)))


def bk_probe_pipe(kind: int, iters: int, grid: int, block: int, sink, stream=None):
    """Launch a pipe-rate probe (0 FP64 FMA, 1 FP32 FMA, 2 MUFU ex2, 3 FP64 -> FP32
    conversion, 4 FP32 -> FP64 conversion); the caller times it.  Returns the
    number of operations the launch performs."""
    torch = _torch()
    _dev(sink, "sink", torch.float64)
    if sink.numel() < grid * block:
        raise ValueError("sink needs grid * block elements")
    _check(lib().bk_probe_pipe(int(kind), int(iters), int(grid), int(block), _ptr(sink),
                               _stream_ptr(stream)))
    return grid * block * iters * 8


MATH_PROBE_FNS = {"exp": 0, "log": 1, "exp2s_node": 2, "exp2s_neg": 3, "round_rem": 4,
                  "two_cosh": 5, "sqrt": 6, "exp_acc": 7, "exp_units": 8,
                  "log_parts": 9, "sqrt_int": 10, "exp2s_fix": 11, "one_plus_w": 12,
                  "fix64": 13}


def bk_math_probe(fn, x, stream=None):
    """Evaluate one of the plain form's device math helpers (MATH_PROBE_FNS)
    on a CUDA float64 tensor; "round_rem" returns an (n, 2) tensor of
    (round(v), v - round(v))."""
    torch = _torch()
    _dev(x, "x", torch.float64)
    k = MATH_PROBE_FNS[fn] if isinstance(fn, str) else int(fn)
    x = x.contiguous()
    n = x.numel()
    out = torch.empty(2 * n if k == 4 else n, dtype=torch.float64, device=x.device)
    _check(lib().bk_math_probe(k, _ptr(x), _ptr(out), n, _stream_ptr(stream)))
    return out.view(n, 2) if k == 4 else out.view(x.shape)


# ---------------------------------------------------------------------------
# batched persistent form

#: numpy layout of bk_matern_desc (56 bytes, natural alignment)
DESC_DTYPE = None


def _desc_dtype():
    global DESC_DTYPE
    if DESC_DTYPE is None:
        import numpy as np
        DESC_DTYPE = np.dtype([("locs", "<u8"), ("n", "<i8"), ("sigma2", "<f8"), ("beta", "<f8"),
                               ("nu", "<f8"), ("out", "<u8"), ("ld", "<i8")])
    return DESC_DTYPE


def make_descs(instances, device=None):
    """Pack [(locs (2, n) CUDA f64, sigma2, beta, nu, out (n, ld) CUDA tensor), ...]
    into a device array of bk_matern_desc (a uint8 tensor)."""
    import numpy as np
    torch = _torch()
    arr = np.zeros(len(instances), dtype=_desc_dtype())
    for k, (locs, s2, be, nu, out) in enumerate(instances):
        n = _locs(locs)
        _dev(out, "out")
        if out.dim() != 2 or out.shape[0] != n or out.shape[1] < n:
            raise ValueError(f"instance {k}: out must be (n, ld) with ld >= n")
        arr[k] = (locs.data_ptr(), n, float(s2), float(be), float(nu), out.data_ptr(), out.shape[1])
    dev = device or (instances[0][0].device if instances else torch.device("cuda"))
    return torch.from_numpy(arr.view(np.uint8).copy()).to(dev)


class BatchedPlan:
    """Work list and launch shape for a fixed list of instance sizes."""

    def __init__(self, sizes, dtype=None, opts: Optional[bk_opts] = None):
        import numpy as np
        torch = _torch()
        self.sizes = np.ascontiguousarray(np.asarray(sizes, dtype=np.int64))
        self.dtype_code = _dtype_code(dtype or torch.float64)
        self.count = int(self.sizes.size)
        self._opts = opts  # keeps the counters pointer alive with the plan
        h = ctypes.c_void_p()
        optp = ctypes.byref(opts) if opts is not None else None
        _check(lib().bk_batched_plan_create(ctypes.byref(h), self.sizes.ctypes.data_as(ctypes.c_void_p),
                                            self.count, self.dtype_code, optp))
        self.handle = h

    def info(self) -> dict:
        t, w, c, ch, tu = (ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(),
                           ctypes.c_int())
        _check(lib().bk_batched_plan_info(self.handle, ctypes.byref(t), ctypes.byref(w),
                                          ctypes.byref(c), ctypes.byref(ch), ctypes.byref(tu)))
        return {"total_tiles": t.value, "warps": w.value, "ctas_per_sm": c.value,
                "chunk": ch.value, "tuned": bool(tu.value)}

    def autotune(self, d_descs, sample_tiles: int = 0, stream=None):
        _check(lib().bk_batched_autotune(self.handle, _ptr(d_descs), int(sample_tiles),
                                         _stream_ptr(stream)))
        return self.info()

    def close(self):
        if getattr(self, "handle", None):
            lib().bk_batched_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bk_matern_batched(d_descs, plan: BatchedPlan, stream=None):
    """All instances of `plan` in one persistent launch (graph-capturable)."""
    torch = _torch()
    _dev(d_descs, "d_descs", torch.uint8)
    if d_descs.numel() != plan.count * _desc_dtype().itemsize:
        raise ValueError("d_descs does not hold plan.count descriptors")
    _check(lib().bk_matern_batched(_ptr(d_descs), plan.count, plan.dtype_code, plan.handle,
                                   _stream_ptr(stream)))


#: most instances bk_matern_batched_static accepts (its scratch is a fixed array)
STATIC_MAX_INSTANCES = 4096


def bk_matern_batched_static(d_descs, count: int, dtype=None, stream=None):
    """bk_matern_batched without a plan and without any allocation, for
    callers that cannot allocate device memory at this point (see bk.h).
    At most STATIC_MAX_INSTANCES instances; calls that overlap on the GPU
    race on the shared scratch, so order them."""
    torch = _torch()
    _dev(d_descs, "d_descs", torch.uint8)
    if d_descs.numel() != int(count) * _desc_dtype().itemsize:
        raise ValueError("d_descs does not hold `count` descriptors")
    code = _dtype_code(dtype or torch.float64)
    _check(lib().bk_matern_batched_static(_ptr(d_descs), int(count), code, _stream_ptr(stream)))


# ---------------------------------------------------------------------------
# learned window

N_MLP_PARAMS = 8772


class LearnedWindow:
    """The window network (bk_learned): training, inference, checkpoints."""

    def __init__(self, seed: int = 0, path: Optional[str] = None):
        h = ctypes.c_void_p()
        _check(lib().bk_learned_create(ctypes.byref(h), ctypes.c_uint64(seed)))
        self.handle = h
        if path is not None:
            self.load(path)

    def train(self, x, nu, labels, steps: int, batch: int = 8192, lr: float = 2e-3,
              seed: int = 1, loss=None, stream=None):
        torch = _torch()
        for t, name in ((x, "x"), (nu, "nu"), (labels, "labels")):
            _dev(t, name, torch.float64)
        n = x.numel()
        if labels.numel() != 6 * n or nu.numel() != n:
            raise ValueError("labels must be (n, 6) and nu (n,)")
        if loss is not None:
            _dev(loss, "loss", torch.float32)
            if loss.numel() < steps:
                raise ValueError("loss needs `steps` entries")
        _check(lib().bk_learned_train(self.handle, _ptr(x), _ptr(nu), _ptr(labels), n, int(steps),
                                      int(batch), float(lr), ctypes.c_uint64(seed), _ptr(loss),
                                      _stream_ptr(stream)))

    def grad(self, x, nu, labels, stream=None):
        """(gradient[8772], loss) of the full-batch loss over the given samples."""
        torch = _torch()
        n = x.numel()
        g = torch.empty(N_MLP_PARAMS, dtype=torch.float32, device=x.device)
        loss = torch.zeros(1, dtype=torch.float32, device=x.device)
        _check(lib().bk_learned_grad(self.handle, _ptr(x), _ptr(nu), _ptr(labels), n, _ptr(g),
                                     _ptr(loss), _stream_ptr(stream)))
        return g, loss

    def infer(self, x, nu, stream=None):
        torch = _torch()
        out = torch.empty((x.numel(), 4), dtype=torch.float32, device=x.device)
        _check(lib().bk_learned_infer(self.handle, _ptr(x), _ptr(nu), _ptr(out), x.numel(),
                                      _stream_ptr(stream)))
        return out

    def params(self, new=None):
        import numpy as np
        cur = np.empty(N_MLP_PARAMS, dtype=np.float32)
        setp = None
        if new is not None:
            new = np.ascontiguousarray(np.asarray(new, dtype=np.float32))
            setp = new.ctypes.data_as(ctypes.c_void_p)
        _check(lib().bk_learned_params(self.handle, cur.ctypes.data_as(ctypes.c_void_p), setp))
        return cur

    def stats(self, new=None):
        import numpy as np
        cur = np.empty(8, dtype=np.float32)
        setp = None
        if new is not None:
            new = np.ascontiguousarray(np.asarray(new, dtype=np.float32))
            setp = new.ctypes.data_as(ctypes.c_void_p)
        _check(lib().bk_learned_stats(self.handle, cur.ctypes.data_as(ctypes.c_void_p), setp))
        return cur

    def set_margins(self, rel: float, abs_margin: float):
        _check(lib().bk_learned_set_margins(self.handle, float(rel), float(abs_margin)))

    def set_train_path(self, path: int):
        """BK_TRAIN_TENSOR (tcgen05 MMAs, the default) or BK_TRAIN_SIMT."""
        _check(lib().bk_learned_set_train_path(self.handle, int(path)))

    def save(self, path: str):
        _check(lib().bk_learned_save(self.handle, path.encode()))

    def load(self, path: str):
        _check(lib().bk_learned_load(self.handle, path.encode()))

    def close(self):
        if getattr(self, "handle", None):
            lib().bk_learned_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
