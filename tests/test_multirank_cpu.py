"""The multi-rank host logic of bench.py on CPU: two gloo ranks (weak
scaling, no collective on the data path) agree on the slowest rank's time and
on the whole-job rate computed from it."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", init_method="env://")
    try:
        bench.barrier(w)
        own_ms = 100.0 + 50.0 * r            # each rank's own timed region
        ms = bench.max_over_ranks(own_ms, w, torch.device("cpu"))
        units = 3 * 40 * 40                  # this rank's entries per step
        out[r] = (r, w, local, ms, bench.job_rate(w, 5, units, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_and_count_all_units():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        rank, w, local, ms, rate = res[r]
        assert (rank, w, local) == (r, world, r)
        assert ms == 150.0                   # the slowest rank's time on every rank
        assert rate == pytest.approx(world * 5 * 3 * 40 * 40 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, None) == 12.5
    assert bench.job_rate(1, 2, 1000, 500.0) == pytest.approx(4000.0)
