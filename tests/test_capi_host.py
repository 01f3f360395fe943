"""CPU-only checks of the C-ABI library: it loads, exports every symbol the
header declares, and rejects bad arguments on the host before any launch.
No kernel runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    bk.build()
    return bk.lib()


def header_functions():
    text = open(os.path.join(ROOT, "include", "bk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bk_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = header_functions()
    assert names, "no declarations parsed"
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, f"not exported: {missing}"
    assert sorted(bk.EXPORTS) == names


def test_version_and_status_strings(L):
    assert "sm_103a" in bk.version()
    assert L.bk_status_string(1) == b"BK_ERR_INVALID_ARG"


def test_opts_default(L):
    o = bk.bk_opts()
    L.bk_opts_default(ctypes.byref(o))
    assert (o.window, o.compute, o.fixed_bins, o.fixed_t1, o.d_counters) == (0, 0, 40, 9.0, None)


def test_host_side_argument_checks(L):
    P = ctypes.c_void_p
    fake = P(0x1000)  # never dereferenced: every call below fails its host check
    assert L.bk_eval(fake, fake, fake, -1, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_eval(None, fake, fake, 5, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_eval(None, None, None, 0, None) == bk.BK_OK  # empty input is a no-op
    assert L.bk_eval_ex(fake, fake, fake, None, 7, 5, None, None) == bk.BK_ERR_INVALID_ARG
    # Matern parameters
    for s2, beta, nu in [(-1.0, 0.1, 0.5), (1.0, 0.0, 0.5), (1.0, 0.1, 0.0), (float("nan"), 0.1, 1.0),
                         (1.0, float("inf"), 1.0)]:
        assert L.bk_matern_tile(fake, 4, s2, beta, nu, fake, 4, 0, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_matern_tile(fake, 4, 1.0, 0.1, 0.5, fake, 3, 0, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_matern_tile(fake, 4, 1.0, 0.1, 0.5, fake, 4, 9, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_matern_tile(None, 4, 1.0, 0.1, 0.5, fake, 4, 0, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_matern_tile2(fake, 4, fake, 3, 1.0, 0.1, 0.5, fake, 2, 0, None, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_matern_tile(None, 0, 1.0, 0.1, 0.5, None, 0, 0, None) == bk.BK_OK
    # training path of a window network: a model is required (none is created here)
    assert L.bk_learned_set_train_path(None, bk.BK_TRAIN_TENSOR) == bk.BK_ERR_INVALID_ARG
    assert L.bk_learned_set_train_path(None, bk.BK_TRAIN_SIMT) == bk.BK_ERR_INVALID_ARG
    assert b"ld" in L.bk_last_error() or len(L.bk_last_error()) > 0


def test_option_checks(L):
    fake = ctypes.c_void_p(0x1000)
    o = bk.bk_opts()
    L.bk_opts_default(ctypes.byref(o))
    o.window = 9
    assert L.bk_eval_ex(fake, fake, fake, None, 0, 5, ctypes.byref(o), None) == bk.BK_ERR_INVALID_ARG
    o.window = bk.BK_WIN_FIXED
    o.fixed_bins = 0
    assert L.bk_eval_ex(fake, fake, fake, None, 0, 5, ctypes.byref(o), None) == bk.BK_ERR_INVALID_ARG
    o.fixed_bins = 40
    o.fixed_t1 = 701.0
    assert L.bk_eval_ex(fake, fake, fake, None, 0, 5, ctypes.byref(o), None) == bk.BK_ERR_INVALID_ARG
    o.fixed_t1 = 9.0
    o.compute = bk.BK_F32  # the fixed window is a plain FP64 form
    assert L.bk_eval_ex(fake, fake, fake, None, 0, 5, ctypes.byref(o), None) == bk.BK_ERR_UNSUPPORTED
    # Temme's series: x threshold in [0, 2], plain FP64 only
    L.bk_opts_default(ctypes.byref(o))
    for bad in (-0.1, 2.5, float("nan"), float("inf")):
        o.series_below = bad
        assert L.bk_eval_ex(fake, fake, fake, None, 0, 5, ctypes.byref(o), None) == bk.BK_ERR_INVALID_ARG
    o.series_below = 0.1
    o.compute = bk.BK_F32
    assert L.bk_eval_ex(fake, fake, fake, None, 0, 5, ctypes.byref(o), None) == bk.BK_ERR_UNSUPPORTED
    # n = 0 with valid options is a no-op
    o.compute = bk.BK_F64
    o.window = bk.BK_WIN_FIXED
    assert L.bk_eval_ex(fake, fake, fake, None, 0, 0, ctypes.byref(o), None) == bk.BK_OK
    # the batched plan applies the same checks
    plan = ctypes.c_void_p()
    sizes = (ctypes.c_int64 * 1)(10)
    o.compute = bk.BK_F32
    assert L.bk_batched_plan_create(ctypes.byref(plan), sizes, 1, 0, ctypes.byref(o)) == bk.BK_ERR_UNSUPPORTED


def test_morton_order_matches_generator(L):
    locs = inputs.jittered_grid(5000, seed=21)
    np.testing.assert_array_equal(bk.bk_morton_order(locs), inputs.morton_order(locs))
    # ties keep their input order (stable)
    dup = np.array([[0.5, 0.5, 0.1, 0.5], [0.5, 0.5, 0.1, 0.5]])
    assert list(bk.bk_morton_order(dup)) == [2, 0, 1, 3]


def test_morton_codes_brute_force():
    # the bit interleave agrees with a per-point brute force on a few points
    pts = np.array([[0.0, 1.0, 0.25, 0.999999, 0.5], [0.0, 0.0, 0.75, 0.999999, 0.5]])
    codes = inputs.morton_codes(pts)
    for k in range(pts.shape[1]):
        qx = min(65535, int(pts[0, k] * 65536))
        qy = min(65535, int(pts[1, k] * 65536))
        z = 0
        for b in range(16):
            z |= ((qx >> b) & 1) << (2 * b) | ((qy >> b) & 1) << (2 * b + 1)
        assert int(codes[k]) == z


def test_generators_are_seeded_and_shaped():
    a, b = inputs.kv_pairs(1000, seed=1), inputs.kv_pairs(1000, seed=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[0].min() >= 1e-3 and a[0].max() <= 140 and a[1].min() >= 0.05 and a[1].max() <= 10
    locs = inputs.jittered_grid(20000, seed=2)
    assert locs.shape == (2, 20000)
    assert locs.min() > 0 and locs.max() < 1
    # grid side 142 for n = 20,000: point 143 is the first of the second row
    s = 1 / 142
    assert abs(locs[1, 142] - 1.5 * s) <= 0.4 * s + 1e-15
    inst = inputs.batched_instances(256)
    ns = np.array([i.n for i in inst])
    assert len(inst) == 256 and ns.min() >= 500 and ns.max() <= 8000


def test_batched_host_checks(L):
    fake = ctypes.c_void_p(0x1000)
    h = ctypes.c_void_p()
    sizes = np.array([10, 20], dtype=np.int64)
    sp = sizes.ctypes.data_as(ctypes.c_void_p)
    assert L.bk_batched_plan_create(ctypes.byref(h), sp, 0, 0, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_batched_plan_create(ctypes.byref(h), None, 2, 0, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_batched_plan_create(ctypes.byref(h), sp, 2, 5, None) == bk.BK_ERR_INVALID_ARG
    neg = np.array([10, -1], dtype=np.int64)
    assert L.bk_batched_plan_create(ctypes.byref(h), neg.ctypes.data_as(ctypes.c_void_p), 2, 0,
                                    None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_matern_batched(fake, 2, 0, None, None) == bk.BK_ERR_INVALID_ARG
    assert L.bk_batched_plan_destroy(None) == bk.BK_OK
    assert bk._desc_dtype().itemsize == 56


def test_matern_tile_host_checks(L):
    """bk_matern_tile_host: the workspace size and the host-side argument
    checks (all fail before any CUDA call)."""
    P = ctypes.c_void_p
    fake = P(0x1000)          # 256-byte aligned, never dereferenced
    odd = P(0x1008)
    need = L.bk_matern_tile_host_workspace(100, bk.BK_F64, 1)
    small = L.bk_matern_tile_host_workspace(100, bk.BK_F64, 0)
    assert need >= 100 * 100 * 8 + small
    assert small >= 2 * 100 * 8 + bk.BK_COSH_TABLE_LEN * 8
    assert L.bk_matern_tile_host_workspace(100, bk.BK_F32, 1) < need
    assert L.bk_matern_tile_host_workspace(-1, bk.BK_F64, 1) == 0
    host = lambda *a: L.bk_matern_tile_host(*a[:9], 0, *a[9:])
    assert host(fake, 100, 1.0, 0.1, 0.5, fake, 100, 0, None, fake, small - 1, None) == bk.BK_ERR_NOMEM
    assert host(fake, 100, 1.0, 0.1, 0.5, fake, 100, 0, None, odd, need, None) == bk.BK_ERR_INVALID_ARG
    assert host(fake, 100, 1.0, 0.1, 0.5, fake, 99, 0, None, fake, need, None) == bk.BK_ERR_INVALID_ARG
    assert host(fake, 100, 1.0, -0.1, 0.5, fake, 100, 0, None, fake, need, None) == bk.BK_ERR_INVALID_ARG
    assert host(None, 100, 1.0, 0.1, 0.5, fake, 100, 0, None, fake, need, None) == bk.BK_ERR_INVALID_ARG
    assert host(fake, 100, 1.0, 0.1, 0.5, fake, 100, 5, None, fake, need, None) == bk.BK_ERR_INVALID_ARG
    assert host(fake, -1, 1.0, 0.1, 0.5, fake, 100, 0, None, fake, need, None) == bk.BK_ERR_INVALID_ARG
    assert host(None, 0, 1.0, 0.1, 0.5, None, 0, 0, None, None, 0, None) == bk.BK_OK
    assert L.bk_matern_tile_host(fake, 100, 1.0, 0.1, 0.5, fake, 100, 0, None, 7, fake, need,
                                 None) == bk.BK_ERR_INVALID_ARG


def test_lanes_option_checks(L):
    P = ctypes.c_void_p
    fake = P(0x1000)
    o = bk.bk_opts()
    L.bk_opts_default(ctypes.byref(o))
    assert o.lanes == 0
    o.compute = bk.BK_F32
    for bad in (3, -1, 16):
        o.lanes = bad
        assert L.bk_eval_ex(fake, fake, fake, None, 1, 5, ctypes.byref(o), None) == bk.BK_ERR_INVALID_ARG
    o.lanes = 0
    o.compute = bk.BK_F64
    best = ctypes.c_int(0)
    assert L.bk_eval_autotune(fake, fake, fake, 0, 5, ctypes.byref(o), None,
                              ctypes.byref(best)) == bk.BK_ERR_UNSUPPORTED
