"""GPU checks of the FP32 precision form against the FP64 oracle.

The form promises relative error <= 1e-5 on K_nu (and on Matern entries that
are representable as normal FP32 numbers); the measured error is asserted
below that.  Entries smaller than 1e-30 (far beyond the correlation range)
are checked in absolute terms only.
"""
import os

import numpy as np
import pytest

import oracle
import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_RTOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


def to_dev(a, dev):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def f32_opts(**kw):
    return bk.make_opts(compute=bk.BK_F32, **kw)


def eval_f32(x, nu, dev, out_dtype=torch.float64):
    out, lout = bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev), out_dtype=out_dtype,
                              opts=f32_opts(), want_log=True)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), lout.cpu().numpy().astype(np.float64)


def test_eval_f32_workload(dev):
    x, nu = inputs.kv_pairs(20_000, seed=1)
    got, lgot = eval_f32(x, nu, dev)
    idx = np.random.default_rng(9).choice(x.size, 4000, replace=False)
    ref, lref = oracle.besselk(x[idx], nu[idx], return_log=True)
    assert np.abs(got[idx] / ref - 1).max() <= F32_RTOL
    assert np.abs(np.expm1(lgot[idx] - lref)).max() <= F32_RTOL


def test_eval_f32_region_grid(dev):
    xs = np.exp(np.linspace(np.log(1e-3), np.log(140.0), 41))
    ns = np.linspace(0.0, 20.0, 41)
    X, V = (a.ravel() for a in np.meshgrid(xs, ns))
    got, lgot = eval_f32(X, V, dev)
    ref, lref = oracle.besselk(X, V, return_log=True)
    assert np.abs(got / ref - 1).max() <= F32_RTOL
    assert np.abs(np.expm1(lgot - lref)).max() <= F32_RTOL


def test_eval_f32_small_x_large_nu(dev):
    # the corner with the peak far out (t* ~ 10): x in [1e-3, 1e-2], nu in [12, 20]
    x, nu = inputs.kv_pairs(6000, seed=77, x_lo=1e-3, x_hi=1e-2, nu_lo=12.0, nu_hi=20.0)
    _, lgot = eval_f32(x, nu, dev)
    _, lref = oracle.besselk(x, nu, return_log=True)
    assert np.abs(np.expm1(lgot - lref)).max() <= 0.5 * F32_RTOL


def test_eval_f32_outside_region_uses_fp64_search(dev):
    # x below 1e-4 or above 1e4 takes the FP64 window search
    x = np.array([3e-5, 5e-5, 2e4, 0.5])
    nu = np.array([0.7, 3.0, 2.0, 45.0])
    _, lgot = eval_f32(x, nu, dev)
    _, lref = oracle.besselk(x, nu, return_log=True)
    assert np.abs(np.expm1(lgot - lref)).max() <= F32_RTOL


def test_eval_f32_counters_and_edges(dev):
    x = np.array([0.0, -2.0, np.inf, 1.0])
    nu = np.array([1.0, 1.0, 1.0, 2.5])
    got, _ = eval_f32(x, nu, dev)
    assert np.isposinf(got[0]) and np.isnan(got[1]) and got[2] == 0.0
    assert abs(got[3] / oracle.besselk(1.0, 2.5) - 1) <= F32_RTOL
    xs, ns = inputs.kv_pairs(1000, seed=4)
    ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
    bk.bk_eval_ex(to_dev(xs, dev), to_dev(ns, dev), opts=f32_opts(counters=ctr))
    torch.cuda.synchronize()
    c = ctr.cpu().numpy()
    assert c[bk.BK_CTR_EVALS] == 1000 and c[bk.BK_CTR_FAIL] == 0
    assert c[bk.BK_CTR_NODES] < 1000 * 40  # eps = 2^-23 window, tol 2e-7: ~13 nodes


def check_entries(got, want, rtol=F32_RTOL):
    big = np.abs(want) >= 1e-30
    rel = np.abs(got[big] / want[big] - 1)
    assert rel.max() <= rtol, f"max rel {rel.max():.3e}"
    assert np.abs(got - want).max() <= rtol * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("n", [1, 33, 97])
@pytest.mark.parametrize("nu", [0.5, 1.7, 3.2])
def test_matern_f32_small(dev, n, nu):
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=300 + n))
    out = torch.full((n, n), float("nan"), dtype=torch.float32, device=dev)
    bk.bk_matern_tile(to_dev(locs, dev), 1.4, 0.05, nu, out=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    want = oracle.matern_block(locs, locs, 1.4, 0.05, nu)
    check_entries(got.T, want)
    assert np.array_equal(got, got.T)
    assert np.all(np.diag(got) == np.float32(1.4))


def test_matern_f32_block_and_f64_output(dev):
    l1 = inputs.jittered_grid(50, seed=61)
    l2 = inputs.jittered_grid(70, seed=62)
    out = bk.bk_matern_tile2(to_dev(l1, dev), to_dev(l2, dev), 1.0, 0.1, 1.3, dtype=torch.float64,
                             opts=f32_opts())
    torch.cuda.synchronize()
    check_entries(out.cpu().numpy().T, oracle.matern_block(l1, l2, 1.0, 0.1, 1.3))


def c3_nu():
    # the precision workload draws nu ~ U(0.3, 3.5) once per run (seed 5)
    return float(np.random.default_rng(5).uniform(0.3, 3.5))


def test_matern_f32_full_size_40000(dev):
    """n = 40,000 on a 200 x 200 jittered grid, beta = 0.05, FP32 output
    (6.4 GB): a 20,000-entry oracle sample with near-diagonal pairs, and every
    entry against the parity-checked FP64 form, slab by slab."""
    n, beta, nu = 40_000, 0.05, c3_nu()
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=4))
    L = to_dev(locs, dev)
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    bk.bk_matern_tile(L, 1.0, beta, nu, out=out)
    torch.cuda.synchronize()
    I, J = inputs.entry_sample(n, 20_000, seed=6)
    got = out[torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)].double().cpu().numpy()
    check_entries(got, oracle.matern_entries(locs, I, J, 1.0, beta, nu))
    worst_rel, worst_abs = 0.0, 0.0
    slab = 2000
    for c0 in range(0, n, slab):
        ref = bk.bk_matern_tile2(L, L[:, c0:c0 + slab].contiguous(), 1.0, beta, nu,
                                 opts=bk.make_opts(compute=bk.BK_F64))
        g = out[c0:c0 + slab, :].double()
        big = ref.abs() >= 1e-30
        worst_rel = max(worst_rel, float(((g - ref).abs() / ref.abs())[big].max()))
        worst_abs = max(worst_abs, float((g - ref).abs().max()))
        del ref, g, big
    assert worst_rel <= F32_RTOL and worst_abs <= F32_RTOL
    del out
    torch.cuda.empty_cache()


def test_matern_f32_cholesky_8000(dev):
    """Cholesky of the n = 8,000 FP32 matrix (first 8,000 of the 200 x 200
    grid in Morton order, beta = 0.05).  The FP32 matrix must factor whenever
    the FP32-rounded FP64 matrix does (for nu >= 2.5 neither does: the exact
    matrix is too ill-conditioned for FP32)."""
    beta = 0.05
    locs = inputs.morton_sorted(inputs.jittered_grid(40_000, seed=4))[:, :8000].copy()
    L = to_dev(locs, dev)
    for nu in (0.5, 1.5, c3_nu()):
        m32 = torch.empty((8000, 8000), dtype=torch.float32, device=dev)
        bk.bk_matern_tile(L, 1.0, beta, nu, out=m32)
        m64 = torch.empty((8000, 8000), dtype=torch.float64, device=dev)
        bk.bk_matern_tile(L, 1.0, beta, nu, out=m64)
        torch.cuda.synchronize()
        _, info32 = torch.linalg.cholesky_ex(m32)
        _, info_ref = torch.linalg.cholesky_ex(m64.float())
        if int(info_ref) == 0:
            assert int(info32) == 0, f"nu={nu}: FP32 matrix failed where the rounded FP64 one factors"
        if nu <= 1.5:
            assert int(info32) == 0


def test_default_form_follows_output_dtype(dev):
    """Without options, FP32 output selects the FP32 precision form (the C
    entry points' default for a NULL options pointer, mirrored by the
    binding): the same bits as asking for compute = BK_F32 explicitly, and
    not the plain form's FP32-rounded matrix."""
    n = 500
    L = torch.as_tensor(inputs.morton_sorted(inputs.jittered_grid(n, seed=251)), device=dev)
    default = bk.bk_matern_tile(L, 1.0, 0.1, 1.3, dtype=torch.float32)
    f32 = bk.bk_matern_tile(L, 1.0, 0.1, 1.3, dtype=torch.float32,
                            opts=bk.make_opts(compute=bk.BK_F32))
    plain = bk.bk_matern_tile(L, 1.0, 0.1, 1.3, dtype=torch.float32,
                              opts=bk.make_opts(compute=bk.BK_F64))
    torch.cuda.synchronize()
    assert torch.equal(default, f32)
    assert not torch.equal(default, plain)
    d2 = bk.bk_matern_tile2(L, L, 1.0, 0.1, 1.3, dtype=torch.float32)
    torch.cuda.synchronize()
    assert torch.equal(d2, f32)



@pytest.mark.parametrize("nu", [0.5, 1.7, 3.2])
def test_matern_f32_small_distances(dev, nu):
    """Entries at r << beta (x down to 1e-6), where nu log x and log K_nu(x)
    grow and cancel in the normalisation: both FP32 forms within 1e-5 of the
    oracle."""
    rng = np.random.default_rng(31)
    n = 150
    locs = 0.5 + 1e-3 * rng.random((2, n))
    locs[:, 1] = locs[:, 0] + 1e-7   # a pair at r ~ 1.4e-7 (x ~ 1.4e-6)
    locs[:, 2] = locs[:, 0] + 3e-5
    locs = np.ascontiguousarray(locs)
    want = oracle.matern_block(locs, locs, 1.3, 0.1, nu)
    L = to_dev(locs, dev)
    net = bk.LearnedWindow(path=os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), "paper_2502_00356_gb300", "weights", "window_mlp.bkw"))
    for opts in (bk.make_opts(compute=bk.BK_F32), bk.make_opts(learned=net)):
        got = bk.bk_matern_tile(L, 1.3, 0.1, nu, dtype=torch.float32, opts=opts)
        torch.cuda.synchronize()
        check_entries(got.cpu().numpy().astype(np.float64).T, want)


def test_zero_sigma2_gives_zero_matrix(dev):
    """sigma^2 = 0 (allowed by the C-ABI): every entry, the diagonal included,
    is 0 in every form and output type."""
    L = to_dev(inputs.morton_sorted(inputs.jittered_grid(70, seed=33)), dev)
    net = bk.LearnedWindow(path=os.path.join(os.path.dirname(os.path.dirname(
        os.path.abspath(__file__))), "paper_2502_00356_gb300", "weights", "window_mlp.bkw"))
    for dtype in (torch.float64, torch.float32):
        for opts in (None, bk.make_opts(compute=bk.BK_F32), bk.make_opts(learned=net)):
            m = bk.bk_matern_tile(L, 0.0, 0.1, 1.7, dtype=dtype, opts=opts)
            torch.cuda.synchronize()
            assert bool((m == 0).all())
