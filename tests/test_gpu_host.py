"""bk_matern_tile_host: the Matern matrix delivered to host memory, either
stored directly by the tile writer into host memory the device can address
(page-locked, and on GB300 pageable memory too), or staged: generated in
panels of block-columns in a device workspace whose copies overlap the later
panels.  Every entry is computed by the same tile writer as
bk_matern_tile, so the host matrix must equal the device one bit for bit (in
either way, whatever the panel boundaries), and the oracle within the plain
form's 1e-10."""
import os

import numpy as np
import pytest

import oracle
import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CKPT = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2502_00356_gb300", "weights", "window_mlp.bkw")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


def host_matrix(locs_h, nu, dtype, ld=None, pinned=True, staged=False, opts=None, sigma2=1.0,
                beta=0.1):
    n = locs_h.shape[1]
    ld = ld or n
    out = torch.full((n, ld), float("nan"), dtype=dtype, pin_memory=pinned)
    work = torch.empty(bk.matern_tile_host_workspace(n, dtype, staged=staged),
                       dtype=torch.uint8, device="cuda")
    bk.bk_matern_tile_host(torch.from_numpy(locs_h), sigma2, beta, nu, out, work, opts=opts,
                           staged=staged)
    torch.cuda.synchronize()
    return out


def device_matrix(locs_h, nu, dtype, dev, opts=None, sigma2=1.0, beta=0.1):
    L = torch.as_tensor(locs_h, device=dev)
    out = bk.bk_matern_tile(L, sigma2, beta, nu, dtype=dtype, opts=opts)
    torch.cuda.synchronize()
    return out.cpu()


@pytest.mark.parametrize("n", [1, 2, 33, 700, 2100])
@pytest.mark.parametrize("dtype", ["float64", "float32"])
@pytest.mark.parametrize("pinned,staged", [(True, False), (False, False), (True, True),
                                           (False, True)])
def test_host_equals_device_bitwise(dev, n, dtype, pinned, staged):
    dt = getattr(torch, dtype)
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=2))
    got = host_matrix(locs, 1.5, dt, pinned=pinned, staged=staged)
    want = device_matrix(locs, 1.5, dt, dev)
    assert torch.equal(got, want)


@pytest.mark.parametrize("staged", [False, True])
def test_host_padding_pageable_and_two_calls(dev, staged):
    """ld > n leaves the padding untouched; a pageable output works; a second
    call with another nu into the same buffers gives that nu's matrix."""
    n, ld = 1000, 1013
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=5))
    work = torch.empty(bk.matern_tile_host_workspace(n, staged=staged), dtype=torch.uint8,
                       device=dev)
    out = torch.full((n, ld), float("nan"), dtype=torch.float64)  # pageable
    for nu in (0.5, 2.3):
        bk.bk_matern_tile_host(torch.from_numpy(locs), 1.0, 0.1, nu, out, work, staged=staged)
        torch.cuda.synchronize()
        assert torch.equal(out[:, :n], device_matrix(locs, nu, torch.float64, dev))
        assert bool(torch.isnan(out[:, n:]).all())


def test_host_against_oracle(dev):
    n = 300
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=6))
    got = host_matrix(locs, 2.3, torch.float64, sigma2=1.7, beta=0.07).numpy()
    want = oracle.matern_block(locs, locs, 1.7, 0.07, 2.3)
    assert np.abs(got.T - want).max() <= 1e-10


def test_host_learned_form(dev):
    net = bk.LearnedWindow(path=CKPT)
    n = 1500
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=7))
    opts = bk.make_opts(learned=net)
    want = device_matrix(locs, 1.7, torch.float32, dev, opts=opts)
    for staged in (False, True):
        got = host_matrix(locs, 1.7, torch.float32, opts=opts, staged=staged)
        assert torch.equal(got, want)


def test_host_workspace_too_small(dev):
    """The direct way needs only the small workspace; the staged way needs
    room for the matrix."""
    n = 64
    locs = torch.from_numpy(inputs.jittered_grid(n, seed=2))
    small = bk.matern_tile_host_workspace(n, staged=False)
    pinned = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    work = torch.empty(small - 8, dtype=torch.uint8, device=dev)
    with pytest.raises(bk.BkError) as err:
        bk.bk_matern_tile_host(locs, 1.0, 0.1, 0.5, pinned, work)
    assert err.value.status == bk.BK_ERR_NOMEM
    work = torch.empty(small, dtype=torch.uint8, device=dev)
    bk.bk_matern_tile_host(locs, 1.0, 0.1, 0.5, pinned, work)
    with pytest.raises(bk.BkError) as err:
        bk.bk_matern_tile_host(locs, 1.0, 0.1, 0.5, pinned, work, staged=True)
    assert err.value.status == bk.BK_ERR_NOMEM
    torch.cuda.synchronize()
    assert torch.equal(pinned, device_matrix(locs.numpy(), 0.5, torch.float64, dev))
