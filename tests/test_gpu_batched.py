"""GPU checks of the batched persistent form (one launch for many uneven
matrices with per-instance parameters), including CUDA-graph capture, the
autotuner and the in-kernel descriptor check."""
import numpy as np
import pytest

import oracle
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


def make_batch(instances, dev, dtype):
    items = []
    for inst in instances:
        L = torch.as_tensor(inst.locations(), device=dev)
        out = torch.full((inst.n, inst.n), float("nan"), dtype=dtype, device=dev)
        items.append((L, inst.sigma2, inst.beta, inst.nu, out))
    return items


def same(a, b):
    """Two kernels computing the same entries agree to the form's quadrature
    accuracy: their FMA contraction and Newton stopping points may differ in
    the last bits, and with them the window ends and node counts."""
    a64, b64 = a.double(), b.double()
    rtol = 1e-13 if a.dtype == torch.float64 else 2e-6
    return bool(((a64 - b64).abs() <= rtol * b64.abs() + 1e-300).all())


def single(item, dtype_opts=None):
    L, s2, be, nu, out = item
    ref = torch.empty_like(out)
    bk.bk_matern_tile(L, s2, be, nu, out=ref, opts=dtype_opts)
    return ref


SMALL = [inputs.MaternInstance(n, 500 + k, 0.5 + 0.2 * k, 0.03 + 0.04 * k, 0.4 + 0.45 * k)
         for k, n in enumerate([1, 33, 64, 100, 2, 257, 31])]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_matches_single_calls_and_oracle(dev, dtype):
    items = make_batch(SMALL, dev, dtype)
    d = bk.make_descs(items)
    plan = bk.BatchedPlan([it[0].shape[1] for it in items], dtype=dtype)
    bk.bk_matern_batched(d, plan)
    torch.cuda.synchronize()
    for inst, item in zip(SMALL, items):
        ref = single(item)
        torch.cuda.synchronize()
        assert same(item[4], ref), f"instance n={inst.n} differs from bk_matern_tile"
        locs = inst.locations()
        I, J = inputs.entry_sample(inst.n, 300, seed=inst.seed)
        got = item[4][torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)].double().cpu().numpy()
        want = oracle.matern_entries(locs, I, J, inst.sigma2, inst.beta, inst.nu)
        tol = 1e-10 if dtype == torch.float64 else 1e-5
        assert np.abs(got - want).max() <= tol * max(1.0, inst.sigma2)


def test_batched_graph_capture_and_replay(dev):
    items = make_batch(SMALL, dev, torch.float32)
    d = bk.make_descs(items)
    plan = bk.BatchedPlan([it[0].shape[1] for it in items], dtype=torch.float32)
    bk.bk_matern_batched(d, plan)  # one eager run before capture
    torch.cuda.synchronize()
    first = [it[4].clone() for it in items]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bk.bk_matern_batched(d, plan)
    for it in items:
        it[4].fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for a, it in zip(first, items):
        assert torch.equal(a, it[4])
    g.replay()  # the counter is reset inside the graph: a second replay works too
    torch.cuda.synchronize()
    for a, it in zip(first, items):
        assert torch.equal(a, it[4])


def test_batched_fp64_replay_follows_new_parameters(dev):
    """The FP64 plan's per-instance tables of e^{-2 nu h} are filled from
    the descriptors at every launch: a captured graph replayed after the
    descriptors' nu (and beta, sigma2) changed in place gives the single-call
    results for the new parameters."""
    items = make_batch(SMALL, dev, torch.float64)
    d = bk.make_descs(items)
    plan = bk.BatchedPlan([it[0].shape[1] for it in items], dtype=torch.float64)
    bk.bk_matern_batched(d, plan)  # one eager run before capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bk.bk_matern_batched(d, plan)
    for shift in (0.0, 0.37, 1.9):
        changed = [(L, s2 * (1 + shift), be * (1 + 0.5 * shift), nu + shift, out)
                   for (L, s2, be, nu, out) in items]
        d.copy_(bk.make_descs(changed))
        for it in items:
            it[4].fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for it in changed:
            assert same(it[4], single(it)), f"nu={it[3]} differs after replay"


def test_batched_autotune_keeps_results(dev, tmp_path, monkeypatch):
    monkeypatch.setenv("BK_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    items = make_batch(SMALL, dev, torch.float64)
    d = bk.make_descs(items)
    sizes = [it[0].shape[1] for it in items]
    plan = bk.BatchedPlan(sizes, dtype=torch.float64)
    info = plan.autotune(d)
    assert info["tuned"] and info["warps"] in (4, 8) and info["ctas_per_sm"] >= 1
    for it in items:
        it[4].fill_(float("nan"))
    bk.bk_matern_batched(d, plan)
    torch.cuda.synchronize()
    for it in items:
        assert same(it[4], single(it))
    # a new plan for the same layout picks the cached shape
    plan2 = bk.BatchedPlan(sizes, dtype=torch.float64)
    assert plan2.info()["tuned"] and plan2.info()["warps"] == info["warps"]
    assert (tmp_path / "tune.txt").exists()


def test_batched_skips_mismatched_descriptor(dev):
    items = make_batch(SMALL[:3], dev, torch.float64)
    ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
    plan = bk.BatchedPlan([1, 40, 64], dtype=torch.float64, opts=bk.make_opts(counters=ctr))
    d = bk.make_descs(items)  # instance 1 has n = 33, the plan says 40
    bk.bk_matern_batched(d, plan)
    torch.cuda.synchronize()
    assert int(ctr[bk.BK_CTR_FAIL]) >= 1
    assert bool(torch.isnan(items[1][4]).all())  # skipped: untouched
    assert same(items[2][4], single(items[2]))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_batched_sweep_256(dev, dtype):
    """The sweep workload: 256 matrices, n log-uniform in [500, 8000],
    sigma^2 ~ U[0.5, 2], beta ~ U[0.02, 0.3], nu ~ U[0.3, 3]; one launch.
    Every instance is compared on sampled entries with the oracle, and three
    instances in full with single-matrix calls."""
    insts = inputs.batched_instances(256)
    items = make_batch(insts, dev, dtype)
    d = bk.make_descs(items)
    plan = bk.BatchedPlan([i.n for i in insts], dtype=dtype)
    bk.bk_matern_batched(d, plan)
    torch.cuda.synchronize()
    tol = 1e-10 if dtype == torch.float64 else 1e-5
    worst = 0.0
    for k, (inst, item) in enumerate(zip(insts, items)):
        I, J = inputs.entry_sample(inst.n, 24, seed=900 + k)
        got = item[4][torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)].double().cpu().numpy()
        want = oracle.matern_entries(inst.locations(), I, J, inst.sigma2, inst.beta, inst.nu)
        worst = max(worst, float(np.abs(got - want).max() / inst.sigma2))
    assert worst <= tol
    for k in (0, 100, 255):
        assert same(items[k][4], single(items[k]))
    del items, d
    torch.cuda.empty_cache()
