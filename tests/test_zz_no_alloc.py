"""bk_matern_batched_static: the batched Matern writer for callers that
cannot allocate device memory where they build their matrices (code running
under a framework that owns all device memory through its own pool, or a
real-time service that forbids allocation after start-up).  It needs no plan
and allocates nothing; its scratch is a fixed array inside the library.

Checked through the C-ABI against the plan-based bk_matern_batched on two
calls in a row with different batches (the second call must not see the
first call's leftover work list or counter), plus an FP32 call and the
host-side size limit.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import paper_2502_00356_gb300 as bk
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F64_ATOL = 1e-10  # the FP64 Matern tolerance of the parity tests
F32_RTOL = 1e-5   # the FP32 form's tolerance

BATCH_A = [inputs.MaternInstance(n, 700 + k, 0.6 + 0.3 * k, 0.04 + 0.03 * k, 0.5 + 0.6 * k)
           for k, n in enumerate([65, 1, 200, 31, 96])]
BATCH_B = [inputs.MaternInstance(n, 800 + k, 1.5 - 0.1 * k, 0.2 - 0.02 * k, 2.4 - 0.3 * k)
           for k, n in enumerate([130, 7, 33, 64, 257, 2, 90])]


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


def batch(instances, dev, dtype):
    items = []
    for inst in instances:
        L = torch.as_tensor(inst.locations(), device=dev)
        out = torch.full((inst.n, inst.n), float("nan"), dtype=dtype, device=dev)
        items.append((L, inst.sigma2, inst.beta, inst.nu, out))
    return items


def with_plan(instances, dev, dtype):
    """Reference: the existing plan-based entry point."""
    items = batch(instances, dev, dtype)
    plan = bk.BatchedPlan([i.n for i in instances], dtype=dtype)
    bk.bk_matern_batched(bk.make_descs(items), plan)
    torch.cuda.synchronize()
    return [it[4] for it in items]


def static_call(instances, dev, dtype):
    items = batch(instances, dev, dtype)
    bk.bk_matern_batched_static(bk.make_descs(items), len(items), dtype=dtype)
    torch.cuda.synchronize()
    return [it[4] for it in items]


def test_static_matches_plan_two_calls_in_a_row(dev):
    ref_a = with_plan(BATCH_A, dev, torch.float64)
    ref_b = with_plan(BATCH_B, dev, torch.float64)
    got_a = static_call(BATCH_A, dev, torch.float64)   # first call
    got_b = static_call(BATCH_B, dev, torch.float64)   # second call, other layout
    for got, ref in list(zip(got_a, ref_a)) + list(zip(got_b, ref_b)):
        assert not bool(torch.isnan(got).any())
        assert float((got - ref).abs().max()) <= F64_ATOL


def test_static_fp32(dev):
    ref = with_plan(BATCH_B, dev, torch.float32)
    got = static_call(BATCH_B, dev, torch.float32)
    for g, r in zip(got, ref):
        assert not bool(torch.isnan(g).any())
        assert float(((g.double() - r.double()).abs() / r.double().abs().clamp_min(1e-30)).max()) <= F32_RTOL


def test_static_rejects_too_many_instances(dev):
    items = batch(BATCH_A[:1], dev, torch.float64)
    d = bk.make_descs(items)
    big = bk.STATIC_MAX_INSTANCES + 1
    d_big = torch.zeros(big * d.numel(), dtype=torch.uint8, device=dev)
    with pytest.raises(bk.BkError) as err:
        bk.bk_matern_batched_static(d_big, big)
    assert err.value.status == bk.BK_ERR_INVALID_ARG
    assert "4096" in str(err.value)


def test_static_skips_an_invalid_descriptor(dev):
    """An invalid descriptor (beta < 0) is skipped without a report: its
    NaN-filled output stays NaN and the other instances still match."""
    ref = with_plan(BATCH_B, dev, torch.float64)
    items = batch(BATCH_B, dev, torch.float64)
    bad = 2
    L, s2, _, nu, out = items[bad]
    items[bad] = (L, s2, -0.1, nu, out)
    bk.bk_matern_batched_static(bk.make_descs(items), len(items), dtype=torch.float64)
    torch.cuda.synchronize()
    for k, (it, r) in enumerate(zip(items, ref)):
        if k == bad:
            assert bool(torch.isnan(it[4]).all())
        else:
            assert float((it[4] - r).abs().max()) <= F64_ATOL


def test_static_call_allocates_no_device_memory(dev):
    """Free device memory (cudaMemGetInfo) is the same before and after a
    call larger than any before it, once both forms' kernels are loaded."""
    small = batch(BATCH_A, dev, torch.float64)
    small32 = batch(BATCH_A, dev, torch.float32)
    big = [inputs.MaternInstance(n, 900 + k, 1.0, 0.1, 0.7 + 0.2 * k)
           for k, n in enumerate([1500, 900, 2100, 64, 700])]
    big64 = batch(big, dev, torch.float64)
    big32 = batch(big, dev, torch.float32)
    descs = [bk.make_descs(x) for x in (small, small32, big64, big32)]
    bk.bk_matern_batched_static(descs[0], len(small), dtype=torch.float64)  # loads the kernels
    bk.bk_matern_batched_static(descs[1], len(small32), dtype=torch.float32)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    bk.bk_matern_batched_static(descs[2], len(big64), dtype=torch.float64)
    bk.bk_matern_batched_static(descs[3], len(big32), dtype=torch.float32)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert not bool(torch.isnan(big64[2][4]).any())
