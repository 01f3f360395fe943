"""GPU checks of bk_gaussian_loglik (blocked FP64 Cholesky, log det and the
forward substitution that turn a generated Matern matrix into the Gaussian
log-likelihood of observations), against numpy's LAPACK on the same
matrices and on the closed-form Matern matrix of nu = 1/2."""
import math

import numpy as np
import pytest

import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


def ref_loglik(A, z):
    L = np.linalg.cholesky(A)
    y = np.linalg.solve(L, z)
    logdet = 2.0 * np.log(np.diag(L)).sum()
    return L, -0.5 * (y @ y + logdet + len(z) * math.log(2 * math.pi)), logdet, y @ y


@pytest.mark.parametrize("n", [1, 63, 64, 65, 333, 1000])
def test_random_spd_factor_and_loglik(dev, n):
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    z = rng.standard_normal(n)
    ld = n + 3
    a = torch.full((n, ld), 7.0, dtype=torch.float64, device=dev)  # a[j, i] = A[i, j]
    a[:, :n] = torch.as_tensor(A.T.copy(), device=dev)
    upper_before = np.triu(a[:, :n].cpu().numpy().T, 1)
    out = bk.bk_gaussian_loglik(a, torch.as_tensor(z, device=dev))
    torch.cuda.synchronize()
    L, l, logdet, q = ref_loglik(A, z)
    got = a[:, :n].cpu().numpy().T
    assert np.abs(np.tril(got) - L).max() <= 1e-12 * np.abs(L).max()
    assert np.array_equal(np.triu(got, 1), upper_before)   # upper triangle untouched
    assert np.all(a[:, n:].cpu().numpy() == 7.0)           # padding untouched
    o = out.cpu().numpy()
    assert abs(o[0] - l) <= 1e-12 * abs(l) and abs(o[1] - logdet) <= 1e-12 * abs(logdet)
    assert abs(o[2] - q) <= 1e-11 * q


def test_matern_matrix_loglik_matches_closed_form_matrix(dev):
    # nu = 1/2: the Matern covariance is sigma^2 exp(-r/beta) exactly (Sec. III-A
    # with the closed form of K_{1/2}), so the reference matrix needs no oracle call
    n, sigma2, beta, nu = 1500, 1.3, 0.1, 0.5
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=3))
    L = torch.as_tensor(locs, device=dev)
    m = bk.bk_matern_tile(L, sigma2, beta, nu)
    z = np.random.default_rng(5).standard_normal(n)
    ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
    out = bk.bk_gaussian_loglik(m, torch.as_tensor(z, device=dev), opts=bk.make_opts(counters=ctr))
    torch.cuda.synchronize()
    r = np.hypot(locs[0][:, None] - locs[0][None, :], locs[1][:, None] - locs[1][None, :])
    A = sigma2 * np.exp(-r / beta)
    _, l, logdet, q = ref_loglik(A, z)
    o = out.cpu().numpy()
    # the matrices agree to ~1e-14; the likelihood is conditioned by the matrix
    assert abs(o[0] - l) <= 1e-8 * abs(l) and abs(o[1] - logdet) <= 1e-8 * abs(logdet)
    assert int(ctr[bk.BK_CTR_FAIL]) == 0


def test_not_positive_definite_gives_nan(dev):
    n = 130
    A = np.eye(n)
    A[100, 100] = -1.0
    a = torch.as_tensor(A.T.copy(), device=dev)
    ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
    out = bk.bk_gaussian_loglik(a, torch.ones(n, dtype=torch.float64, device=dev),
                                opts=bk.make_opts(counters=ctr))
    torch.cuda.synchronize()
    assert np.all(np.isnan(out.cpu().numpy()[:2]))
    assert int(ctr[bk.BK_CTR_FAIL]) >= 1


def test_empty_and_argument_checks(dev):
    e = torch.empty((0, 0), dtype=torch.float64, device=dev)
    out = torch.full((3,), 5.0, dtype=torch.float64, device=dev)
    bk.bk_gaussian_loglik(e, torch.empty(0, dtype=torch.float64, device=dev), out=out)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 0.0)
    a = torch.eye(4, dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        bk.bk_gaussian_loglik(a, torch.ones(3, dtype=torch.float64, device=dev))
