"""GPU parity of the plain FP64 form against the CPU oracle, through the C-ABI.

Tolerances: K_nu within 1e-10 relative; Matern entries within 1e-10 absolute
(entries lie in (0, sigma^2] with sigma^2 = O(1)).  Sizes span several tiles
with ragged tails; the full-size workloads are checked on sampled entries the
oracle computes one by one, and exhaustively through closed forms.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K_RTOL = 1e-10
M_ATOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


def to_dev(a, dev):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def gpu_eval(x, nu, dev, **kw):
    out = bk.bk_eval(to_dev(x, dev), to_dev(nu, dev), **kw)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def assert_rel(got, want, rtol):
    rel = np.abs(got / want - 1.0)
    i = int(np.argmax(rel))
    assert rel.max() <= rtol, f"max rel {rel.max():.3e} at {i}: got {got[i]!r} want {want[i]!r}"


@pytest.mark.parametrize("n", [1, 31, 129, 1000, 4097])
def test_eval_parity_ragged(dev, n):
    x, nu = inputs.kv_pairs(n, seed=100 + n)
    got = gpu_eval(x, nu, dev)
    assert_rel(got, oracle.besselk(x, nu), K_RTOL)


def test_eval_parity_region_grid(dev):
    # the region of Sec. IV-C: x in [1e-3, 140], nu in (0, 20], plus nu = 0
    xs = np.exp(np.linspace(np.log(1e-3), np.log(140.0), 45))
    ns = np.linspace(0.0, 20.0, 41)
    X, V = (a.ravel() for a in np.meshgrid(xs, ns))
    got = gpu_eval(X, V, dev)
    assert_rel(got, oracle.besselk(X, V), K_RTOL)


def test_eval_full_size_sampled(dev):
    # 100,000 seeded pairs, x log-uniform in [1e-3, 140], nu in [0.05, 10]
    x, nu = inputs.kv_pairs(100_000, seed=1)
    got = gpu_eval(x, nu, dev)
    assert np.all(np.isfinite(got)) and np.all(got > 0)
    idx = np.random.default_rng(5).choice(x.size, 3000, replace=False)
    assert_rel(got[idx], oracle.besselk(x[idx], nu[idx]), K_RTOL)


@pytest.mark.parametrize("n", [1023, 1025, 300_001, 2_000_003])
def test_eval_sorted_chunks_keep_positions(dev, n):
    """The bare-evaluation kernels order each chunk of up to 1,024 pairs by a
    cost bucket before evaluating it and put each result back at its pair's
    position: evaluating the pairs in another order and putting the results
    back agrees to rounding (the 2 cosh h tier of steps off the table's grid
    is voted per warp, so a pair's last bits can depend on its warp-mates; a
    misplaced result would be off by O(1)).  Sizes give blocks with several chunks and ragged last
    chunks; special pairs (0, inf, NaN, negative nu, the series range) are
    mixed in; samples go to the oracle."""
    x, nu = inputs.kv_pairs(n, seed=700 + n % 97)
    rng = np.random.default_rng(n)
    spec = rng.choice(n, min(n, 40), replace=False)
    x[spec[:8]] = 0.0
    x[spec[8:12]] = np.inf
    x[spec[12:16]] = np.nan
    nu[spec[16:24]] *= -1.0
    x[spec[24:]] = 10.0 ** rng.uniform(-6, -3, spec[24:].size)
    opts = bk.make_opts(series_below=0.1)
    X, V = to_dev(x, dev), to_dev(nu, dev)
    got = bk.bk_eval_ex(X, V, opts=opts)[0]
    perm = torch.as_tensor(rng.permutation(n), device=dev)
    got_p = bk.bk_eval_ex(X[perm].contiguous(), V[perm].contiguous(), opts=opts)[0]
    back = torch.empty_like(got_p)
    back[perm] = got_p
    torch.cuda.synchronize()
    a, b = got.cpu().numpy(), back.cpu().numpy()

    def same(u, v, scale):
        # |u - v| within 1e-13 of max(|u|, |scale|): K itself for K, and
        # K (1 + nu/x) for the derivatives, whose values can pass through 0
        fin = np.isfinite(u)
        assert np.array_equal(fin, np.isfinite(v))
        assert np.array_equal(u[~fin], v[~fin], equal_nan=True)
        den = np.maximum(np.abs(u[fin]), np.abs(scale[fin]))
        rel = np.abs(u[fin] - v[fin]) / np.maximum(den, 1e-300)
        assert rel.max(initial=0.0) <= 1e-13, f"max rel {rel.max():.3e}"

    same(a, b, a)
    gk, gdx, gdn = bk.bk_eval_grad(X, V)
    pk, pdx, pdn = bk.bk_eval_grad(X[perm].contiguous(), V[perm].contiguous())
    kk = gk.cpu().numpy()
    with np.errstate(all="ignore"):
        dscale = kk * (1.0 + np.abs(nu) / x)
    for g, p, sc in ((gk, pk, kk), (gdx, pdx, dscale), (gdn, pdn, dscale)):
        q = torch.empty_like(p)
        q[perm] = p
        same(g.cpu().numpy(), q.cpu().numpy(), sc)
    ok = np.isfinite(x) & (x > 0)
    idx = rng.choice(np.flatnonzero(ok), min(2000, int(ok.sum())), replace=False)
    assert_rel(a[idx], oracle.besselk(x[idx], np.abs(nu[idx])), K_RTOL)
    assert np.all(np.isnan(a[spec[12:16]])) and np.all(a[spec[:8]] == np.inf)
    assert np.all(a[spec[8:12]] == 0.0)


def test_eval_node_loop_regions(dev):
    """Both quadrature loops of the plain form and the switch between them:
    the uncentred loop (most windows: the x cosh t recurrence, e^{nu t} as a
    fixed-point running exponent, 1 + e^{-2 nu t} as a fixed-point geometric
    factor) and the centred loop (x cosh t1 > 690, many nodes at nu (t1 -
    t0) small, nu (t1 - t0) > 600, the FP64 search).  Beyond the 1e-10
    requirement, log K must agree with the oracle to 1e-12 + 2e-15 |log K|
    (the rounding of a log assembled from terms as large as |log K|), so that
    an error growing along either loop would show."""
    rng = np.random.default_rng(41)
    m = 4000
    sets = {
        "large x": (np.exp(rng.uniform(np.log(100.0), np.log(3000.0), m)), rng.uniform(0, 30, m)),
        "small nu": (np.exp(rng.uniform(np.log(1e-4), np.log(2.0), m)), rng.uniform(0, 0.03, m)),
        "large nu": (np.exp(rng.uniform(np.log(1e-3), np.log(140.0), m)), rng.uniform(10, 40, m)),
        "region": inputs.kv_pairs(m, seed=42),
    }
    for name, (x, nu) in sets.items():
        for search_f64 in (False, True):
            _, lout = bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev), want_log=True,
                                    opts=bk.make_opts(search_f64=search_f64))
            torch.cuda.synchronize()
            got = lout.cpu().numpy()
            _, want = oracle.besselk(x, nu, return_log=True)
            err = np.abs(got - want)
            bound = 1e-12 + 2e-15 * np.abs(want)
            i = int(np.argmax(err / bound))
            assert np.all(err <= bound), (name, search_f64, x[i], nu[i], err[i])


def test_eval_domain_edges(dev):
    x = np.array([0.0, -1.0, np.nan, np.inf, 2.0, 2.0, 1e-3, 0.5])
    nu = np.array([1.0, 1.0, 1.0, 1.0, -3.3, np.nan, 20.0, 0.0])
    got = gpu_eval(x, nu, dev)
    assert np.isposinf(got[0]) and np.isnan(got[1]) and np.isnan(got[2]) and got[3] == 0.0
    assert abs(got[4] / oracle.besselk(2.0, 3.3) - 1) < K_RTOL
    assert np.isnan(got[5])
    assert abs(got[6] / oracle.besselk(1e-3, 20.0) - 1) < K_RTOL
    assert abs(got[7] / oracle.besselk(0.5, 0.0) - 1) < K_RTOL


def test_eval_empty_and_log_output(dev):
    e = torch.empty(0, dtype=torch.float64, device=dev)
    assert bk.bk_eval(e, e).numel() == 0
    x, nu = inputs.kv_pairs(500, seed=7, nu_hi=20.0)
    out, lout = bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev), want_log=True)
    torch.cuda.synchronize()
    _, lref = oracle.besselk(x, nu, return_log=True)
    err = np.abs(np.expm1(lout.cpu().numpy() - lref))
    assert err.max() < K_RTOL
    out32, _ = bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev), out_dtype=torch.float32)
    torch.cuda.synchronize()
    ref = oracle.besselk(x, nu)
    ok = (ref < 3e38) & (ref > 1.2e-38)  # the FP32 normal range
    assert_rel(out32.cpu().numpy().astype(np.float64)[ok], ref[ok], 1.2e-7)


def test_eval_counters(dev):
    x, nu = inputs.kv_pairs(2000, seed=8)
    counts = {}
    for search_f64 in (False, True):
        ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
        opts = bk.make_opts(counters=ctr, search_f64=search_f64)
        bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev), opts=opts)
        torch.cuda.synchronize()
        c = counts[search_f64] = ctr.cpu().numpy()
        assert c[bk.BK_CTR_EVALS] == 2000 and c[bk.BK_CTR_FAIL] == 0
        assert 2000 * 5 < c[bk.BK_CTR_NODES] < 2000 * 80
    # default: FP32 roots checked in FP64, no FP64 Newton iteration and no
    # window rejected on this set (all points inside the FP32 search region)
    assert counts[False][bk.BK_CTR_ITERS] == 0 and counts[False][bk.BK_CTR_PEAK_ITERS] == 0
    assert counts[False][bk.BK_CTR_FALLBACK] == 0
    # the full FP64 search iterates for every point
    assert counts[True][bk.BK_CTR_ITERS] >= 2000 and counts[True][bk.BK_CTR_PEAK_ITERS] > 0
    assert counts[True][bk.BK_CTR_FALLBACK] == 0
    # both windows enclose the eps-window: node totals agree to a few per cent
    assert abs(counts[True][bk.BK_CTR_NODES] / counts[False][bk.BK_CTR_NODES] - 1) < 0.02


def test_eval_fp32_roots_agree_with_fp64_search(dev):
    """The checked FP32-root window and the FP64 search give the same K_nu
    to quadrature accuracy, inside the FP32 search region (x in [1e-4, 1e4],
    nu <= 40) and outside it (where both take the FP64 search), and both
    match the oracle where it is defined."""
    rng = np.random.default_rng(21)
    x = np.exp(rng.uniform(np.log(1e-6), np.log(1e5), 20_000))
    nu = rng.uniform(0.0, 45.0, 20_000)
    X, V = to_dev(x, dev), to_dev(nu, dev)
    ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
    a, la = bk.bk_eval_ex(X, V, opts=bk.make_opts(counters=ctr), want_log=True)
    b, lb = bk.bk_eval_ex(X, V, opts=bk.make_opts(search_f64=True), want_log=True)
    torch.cuda.synchronize()
    la, lb = la.cpu().numpy(), lb.cpu().numpy()
    assert np.all(np.isfinite(la)) and np.all(np.isfinite(lb))
    # log K is assembled from terms as large as |log K| (~570 at x = 1e-6,
    # nu = 45; ~1e5 at x = 1e5), each rounded to ~1e-16 of its size: compare
    # the logs to 2e-12 plus that conditioning term
    d = np.abs(la - lb)
    i = int(np.argmax(d / (2e-12 + 1e-14 * np.abs(lb))))
    assert d[i] <= 2e-12 + 1e-14 * abs(lb[i]), (x[i], nu[i], la[i], lb[i])
    c = ctr.cpu().numpy()
    assert c[bk.BK_CTR_FAIL] == 0 and c[bk.BK_CTR_FALLBACK] <= 20
    idx = rng.choice(np.flatnonzero(x <= 140.0), 2000, replace=False)
    _, lref = oracle.besselk(x[idx], nu[idx], return_log=True)
    ok = np.isfinite(lref)
    assert np.abs(np.expm1(la[idx][ok] - lref[ok])).max() <= K_RTOL


# ---------------------------------------------------------------------------
# Matern matrices

def gpu_matern(locs, sigma2, beta, nu, dev, dtype=torch.float64, ld=None, opts=None):
    n = locs.shape[1]
    out = torch.full((n, ld or n), float("nan"), dtype=dtype, device=dev)
    bk.bk_matern_tile(to_dev(locs, dev), sigma2, beta, nu, out=out, opts=opts)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n", [1, 2, 33, 70, 130])
@pytest.mark.parametrize("nu", [0.5, 1.37, 2.3])
def test_matern_full_parity(dev, n, nu):
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=200 + n))
    sigma2, beta = 1.3, 0.1
    got = gpu_matern(locs, sigma2, beta, nu, dev)  # got[j, i] = M(i, j)
    want = oracle.matern_block(locs, locs, sigma2, beta, nu)
    assert np.abs(got.T - want).max() <= M_ATOL
    assert np.array_equal(got, got.T)
    assert np.all(np.diag(got) == sigma2)


@pytest.mark.parametrize("nu", [0.5, 2.3, 7.5])
def test_matern_fp64_search_option(dev, nu):
    """bk_opts.search_f64 = 1 (FP64 Newton search for every entry) writes the
    same matrix as the default FP32-root window to rounding."""
    locs = inputs.morton_sorted(inputs.jittered_grid(700, seed=230))
    a = gpu_matern(locs, 1.0, 0.1, nu, dev)
    b = gpu_matern(locs, 1.0, 0.1, nu, dev, opts=bk.make_opts(search_f64=True))
    assert np.abs(a - b).max() <= 1e-12  # two windows, two node counts: quadrature-level agreement


def test_matern_graph_capture(dev):
    """bk_matern_tile captured in a CUDA graph (its per-call table of
    e^{-2 nu h} lives in stream-ordered memory, which capture turns into
    graph allocations) replays to the eager result, twice."""
    n = 700
    L = to_dev(inputs.morton_sorted(inputs.jittered_grid(n, seed=240)), dev)
    eager = torch.empty((n, n), dtype=torch.float64, device=dev)
    bk.bk_matern_tile(L, 1.1, 0.1, 1.5, out=eager)
    torch.cuda.synchronize()
    out = torch.empty_like(eager)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):  # a warm-up on the capture stream
        bk.bk_matern_tile(L, 1.1, 0.1, 1.5, out=out)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bk.bk_matern_tile(L, 1.1, 0.1, 1.5, out=out)
    for _ in range(2):
        out.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, eager)


def test_matern_with_and_without_cosh_table(dev):
    """The C entry point without bk_opts.d_cosh_table computes e^{-2 nu h}
    in the kernel; the Python binding passes a scratch table that a small
    kernel fills by the same arithmetic: the two agree to the last bits."""
    import ctypes
    n = 600
    L = to_dev(inputs.morton_sorted(inputs.jittered_grid(n, seed=241)), dev)
    for nu in (0.5, 1.7, 2.9):
        with_table = bk.bk_matern_tile(L, 1.0, 0.1, nu)
        plain = torch.empty((n, n), dtype=torch.float64, device=dev)
        rc = bk.lib().bk_matern_tile(L.data_ptr(), n, 1.0, 0.1, nu, plain.data_ptr(), n, bk.BK_F64,
                                     torch.cuda.current_stream().cuda_stream or None)
        assert rc == bk.BK_OK
        torch.cuda.synchronize()
        assert float((with_table - plain).abs().max()) <= 1e-15
        assert torch.equal(plain, plain.T)


def test_matern_ld_padding_and_duplicates(dev):
    locs = inputs.jittered_grid(40, seed=31)
    locs[:, 7] = locs[:, 3]
    got = gpu_matern(locs, 1.0, 0.2, 1.1, dev, ld=45)
    assert np.all(np.isnan(got[:, 40:]))  # padding rows of each column untouched
    M = got[:, :40]
    assert M[3, 7] == 1.0 and M[7, 3] == 1.0
    want = oracle.matern_block(locs, locs, 1.0, 0.2, 1.1)
    assert np.abs(M.T - want).max() <= M_ATOL


def test_matern_tile2_block(dev):
    l1 = inputs.jittered_grid(45, seed=41)
    l2 = inputs.jittered_grid(77, seed=42) * 0.8 + 0.1
    out = bk.bk_matern_tile2(to_dev(l1, dev), to_dev(l2, dev), 0.7, 0.15, 1.9)
    torch.cuda.synchronize()
    want = oracle.matern_block(l1, l2, 0.7, 0.15, 1.9)
    assert np.abs(out.cpu().numpy().T - want).max() <= M_ATOL


def test_matern_fp32_output_of_plain_form(dev):
    locs = inputs.morton_sorted(inputs.jittered_grid(100, seed=51))
    got32 = gpu_matern(locs, 1.0, 0.1, 1.5, dev, dtype=torch.float32,
                       opts=bk.make_opts(compute=bk.BK_F64))
    got64 = gpu_matern(locs, 1.0, 0.1, 1.5, dev)
    # the FP32 and FP64 output kernels are separate instantiations: their
    # entries agree to the rounding of FP32 output
    np.testing.assert_allclose(got32, got64, rtol=1.2e-7, atol=0)


def closed_form(z, nu):
    if nu == 0.5:
        return torch.exp(-z)
    if nu == 1.5:
        return (1 + z) * torch.exp(-z)
    raise ValueError(nu)


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.3])
def test_matern_full_size_20000(dev, nu):
    """The n = 20,000 jittered-grid workload (beta = 0.1, sigma^2 = 1): every
    entry against the closed form for nu = 1/2 and 3/2, and a 4,000-entry
    oracle sample (with near-diagonal pairs) for each nu."""
    n, beta = 20_000, 0.1
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=2))
    L = to_dev(locs, dev)
    out = torch.empty((n, n), dtype=torch.float64, device=dev)
    bk.bk_matern_tile(L, 1.0, beta, nu, out=out)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out).all())
    if nu in (0.5, 1.5):
        worst = 0.0
        for c0 in range(0, n, 2000):  # column slabs keep the temporary small
            cols = L[:, c0:c0 + 2000]
            d = torch.sqrt((L[0][:, None] - cols[0][None, :]) ** 2 + (L[1][:, None] - cols[1][None, :]) ** 2)
            ref = closed_form(d / beta, nu)
            worst = max(worst, float((out[c0:c0 + 2000, :].T - ref).abs().max()))
        assert worst <= M_ATOL
    I, J = inputs.entry_sample(n, 4000, seed=6)
    got = out[torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)].cpu().numpy()
    want = oracle.matern_entries(locs, I, J, 1.0, beta, nu)
    assert np.abs(got - want).max() <= M_ATOL
    # symmetry on a sample of transposed pairs
    assert torch.equal(out[torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)],
                       out[torch.as_tensor(I, device=dev), torch.as_tensor(J, device=dev)])
    del out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("nu", [0.5, 1.5, 2.3])
def test_matern_cholesky_4000(dev, nu):
    locs = inputs.morton_sorted(inputs.jittered_grid(4000, seed=3))
    out = torch.empty((4000, 4000), dtype=torch.float64, device=dev)
    bk.bk_matern_tile(to_dev(locs, dev), 1.0, 0.1, nu, out=out)
    torch.cuda.synchronize()
    _, info = torch.linalg.cholesky_ex(out)
    assert int(info) == 0
