"""GPU checks of bk_eval_grad (K, dK/dx, dK/dnu from one quadrature of the
plain FP64 form) against the oracle's derivatives (the integral
differentiated under the sign, pinned by the recurrence identity and DLMF
10.38.7 on the CPU)."""
import numpy as np
import pytest

import oracle
import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


def to_dev(a, dev):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def grad(x, nu, dev, opts=None):
    out = bk.bk_eval_grad(to_dev(x, dev), to_dev(nu, dev), opts=opts)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in out)


def check(got, want):
    k, dx, dn = got
    wk, wx, wn = want
    assert np.abs(k / wk - 1).max() <= RTOL
    assert np.abs(dx / wx - 1).max() <= RTOL
    # dK/dnu vanishes at nu = 0: relative to max(|dK/dnu|, K)
    assert (np.abs(dn - wn) / np.maximum(np.abs(wn), wk)).max() <= RTOL


@pytest.mark.parametrize("n", [1, 37, 1000, 4099])
def test_grad_parity_ragged(dev, n):
    x, nu = inputs.kv_pairs(n, seed=400 + n, nu_hi=20.0)
    check(grad(x, nu, dev), oracle.besselk_grad(x, nu))


def test_grad_region_grid_and_fp64_search(dev):
    xs = np.exp(np.linspace(np.log(1e-3), np.log(140.0), 31))
    ns = np.linspace(0.0, 20.0, 21)
    X, V = (a.ravel() for a in np.meshgrid(xs, ns))
    want = oracle.besselk_grad(X, V)
    ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
    got = grad(X, V, dev, bk.make_opts(counters=ctr))
    check(got, want)
    c = ctr.cpu().numpy()
    assert c[bk.BK_CTR_EVALS] == X.size and c[bk.BK_CTR_FAIL] == 0 and c[bk.BK_CTR_FALLBACK] == 0
    check(grad(X, V, dev, bk.make_opts(search_f64=True)), want)
    assert np.all(got[2][V == 0.0] == 0.0)


def test_grad_consistent_with_eval_and_odd_in_nu(dev):
    x, nu = inputs.kv_pairs(3000, seed=401, nu_hi=20.0)
    k, dx, dn = grad(x, nu, dev)
    k2 = bk.bk_eval(to_dev(x, dev), to_dev(nu, dev)).cpu().numpy()
    assert np.abs(k / k2 - 1).max() <= 1e-12
    km, dxm, dnm = grad(x, -nu, dev)
    assert np.array_equal(km, k) and np.array_equal(dxm, dx) and np.array_equal(dnm, -dn)


def test_grad_domain_and_outputs(dev):
    x = np.array([0.0, np.inf, -1.0, np.nan, 1.0, 2.0])
    nu = np.array([1.0, 1.0, 1.0, 1.0, np.inf, 0.5])
    k, dx, dn = grad(x, nu, dev)
    assert k[0] == np.inf and dx[0] == -np.inf and np.isnan(dn[0])
    assert k[1] == 0.0 and dx[1] == 0.0 and dn[1] == 0.0
    assert np.all(np.isnan(k[2:5])) and np.all(np.isnan(dx[2:5])) and np.all(np.isnan(dn[2:5]))
    want = oracle.besselk_grad(x[5:], nu[5:])
    check((k[5:], dx[5:], dn[5:]), want)
    # outputs may be skipped; empty input is a no-op
    X, V = to_dev(x[5:], dev), to_dev(nu[5:], dev)
    only = torch.empty(1, dtype=torch.float64, device=dev)
    L = bk.lib()
    assert L.bk_eval_grad(bk._ptr(X), bk._ptr(V), None, bk._ptr(only), None, 1, None, None) == 0
    torch.cuda.synchronize()
    assert abs(float(only[0]) / want[1][0] - 1) <= RTOL
    e = torch.empty(0, dtype=torch.float64, device=dev)
    assert all(t.numel() == 0 for t in bk.bk_eval_grad(e, e))


def test_grad_rejects_other_forms(dev):
    x = torch.ones(4, dtype=torch.float64, device=dev)
    for opts in (bk.make_opts(compute=bk.BK_F32), bk.make_opts(series_below=0.1),
                 bk.paper_algorithm2_opts()):
        with pytest.raises(bk.BkError) as e:
            bk.bk_eval_grad(x, x, opts=opts)
        assert e.value.status == bk.BK_ERR_UNSUPPORTED
