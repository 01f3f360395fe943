"""The lane-split quadrature of the FP32 forms' bare evaluations (bk_opts.lanes
= 1, 2, 4, 8; Sec. VI's multi-threaded evaluation of K_nu on the node loop of
Algorithm 2): every lane count must meet the FP32 form's 1e-5 against the
oracle, agree with the others to the rounding of the summation order, count
the same nodes, evaluations and fallbacks, and keep the domain rules."""
import os

import numpy as np
import pytest

import oracle
import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32_RTOL = 1e-5
CROSS_RTOL = 2e-6  # two summation orders of the same FP32 nodes (Kahan sums, ~30 nodes)
CKPT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2502_00356_gb300", "weights", "window_mlp.bkw")
LANES = [1, 2, 4, 8]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def net(dev):
    return bk.LearnedWindow(path=CKPT)


def to_dev(a, dev):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)


def opts_for(form, net, lanes, ctr=None):
    if form == "learned":
        return bk.make_opts(learned=net, lanes=lanes, counters=ctr)
    return bk.make_opts(compute=bk.BK_F32, lanes=lanes, counters=ctr)


def run(x, nu, dev, opts, out_dtype=torch.float32):
    out, lout = bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev), out_dtype=out_dtype, opts=opts,
                              want_log=True)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), lout.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("form", ["search", "learned"])
@pytest.mark.parametrize("out_dtype", ["float32", "float64"])
def test_every_lane_count_matches_the_oracle(dev, net, form, out_dtype):
    n = 4097  # several blocks and a ragged last warp
    x, nu = inputs.kv_pairs(n, seed=21, nu_lo=0.05, nu_hi=20.0)
    idx = np.random.default_rng(22).choice(n, 1500, replace=False)
    _, lref = oracle.besselk(x[idx], nu[idx], return_log=True)
    logs, ctrs = [], []
    for L in LANES:
        ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
        k, lk = run(x, nu, dev, opts_for(form, net, L, ctr), getattr(torch, out_dtype))
        assert np.abs(np.expm1(lk[idx] - lref)).max() <= F32_RTOL
        # K itself where the output type holds it (K_20(1e-3) ~ 1e80 overflows FP32)
        fits = (lref > -80.0) & (lref < 80.0) if out_dtype == "float32" else np.ones_like(lref, bool)
        assert np.abs(k[idx][fits] / np.exp(lref[fits]) - 1).max() <= F32_RTOL
        if out_dtype == "float32":
            assert np.all(np.isposinf(k[idx][lref > 89.0]))  # beyond FP32: +inf, not NaN
            assert not np.any(np.isnan(k))
        logs.append(lk)
        ctrs.append(ctr.cpu().numpy())
    for lk in logs[1:]:  # log K is rounded to the output type: allow 2 of its ulps
        assert np.all(np.abs(lk - logs[0]) <= CROSS_RTOL + 2.4e-7 * np.abs(logs[0]))
    for c in ctrs:
        assert c[bk.BK_CTR_EVALS] == n and c[bk.BK_CTR_FAIL] == 0
        for k in (bk.BK_CTR_NODES, bk.BK_CTR_FALLBACK, bk.BK_CTR_REPAIR, bk.BK_CTR_ITERS):
            assert c[k] == ctrs[0][k]


@pytest.mark.parametrize("n", [1, 31, 33, 130])
@pytest.mark.parametrize("L", LANES)
def test_ragged_sizes(dev, net, n, L):
    x, nu = inputs.kv_pairs(n, seed=23 + n, nu_lo=0.05, nu_hi=20.0)
    _, lref = oracle.besselk(x, nu, return_log=True)
    for form in ("search", "learned"):
        _, lk = run(x, nu, dev, opts_for(form, net, L))
        assert np.abs(np.expm1(lk - lref)).max() <= F32_RTOL


@pytest.mark.parametrize("L", LANES)
def test_fallback_pass_and_domain_edges(dev, L):
    """A zeroed network sends most points to the second (searched-window)
    pass; edge inputs and points outside the FP32 region share the warp."""
    m = bk.LearnedWindow(seed=0, path=CKPT)
    m.params(np.zeros(bk.N_MLP_PARAMS, dtype=np.float32))
    x, nu = inputs.kv_pairs(600, seed=24, nu_hi=20.0)
    x[:6] = [0.0, -1.0, np.inf, np.nan, 3e-5, 2e4]
    nu[:6] = [1.0, 1.0, 1.0, 1.0, 0.7, 2.0]
    ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
    k, lk = run(x, nu, dev, bk.make_opts(learned=m, lanes=L, counters=ctr), torch.float64)
    assert np.isposinf(k[0]) and np.isnan(k[1]) and k[2] == 0.0 and np.isnan(k[3])
    _, lref = oracle.besselk(x[4:], nu[4:], return_log=True)
    assert np.abs(np.expm1(lk[4:] - lref)).max() <= F32_RTOL
    assert ctr.cpu().numpy()[bk.BK_CTR_FALLBACK] > 0.5 * 594


def test_autotune_picks_a_lane_count_that_is_then_used(dev, net):
    x, nu = inputs.kv_pairs(200_000, seed=25, nu_lo=0.05, nu_hi=20.0)
    X, V = to_dev(x, dev), to_dev(nu, dev)
    out = torch.empty(x.size, dtype=torch.float32, device=dev)
    best = bk.bk_eval_autotune(X, V, out, bk.make_opts(learned=net))
    assert best in LANES
    a, _ = bk.bk_eval_ex(X, V, out_dtype=torch.float32, opts=bk.make_opts(learned=net))
    b, _ = bk.bk_eval_ex(X, V, out_dtype=torch.float32, opts=bk.make_opts(learned=net, lanes=best))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    with pytest.raises(bk.BkError) as err:
        bk.bk_eval_autotune(X, V, out, bk.make_opts())  # the FP64 form has no lane split
    assert err.value.status == bk.BK_ERR_UNSUPPORTED
