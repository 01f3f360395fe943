#!/usr/bin/env python3
"""Benchmark of libbesselk's hot path on GB300.

One step = the plain FP64 Matern matrices of the jittered-grid workload
(n = 20,000 locations on a 142 x 142 unit-square grid jittered by
U(-0.4, 0.4) spacing, Morton ordered; sigma^2 = 1, beta = 0.1) for
nu in {0.5, 1.5, 2.3}: three full n x n FP64 matrices (3.2 GB each).
`value` = Matern entries per second over all ranks (weak scaling: every rank
builds its own matrices; no collective on the data path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

`--impl reference` times the CPU oracle (the test-only long-double
implementation) on bounded samples of the same workload on the host cores.
Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "K_ν evals/s, Matérn entries/s (1 GB300): plain FP64 vs learned/FP32, same err"
N_LOC, BETA, SIGMA2, NUS, SEED = 20_000, 0.1, 1.0, (0.5, 1.5, 2.3), 2
WORKLOAD = "matern_jittered_grid_n20000_beta0.1_nu{0.5,1.5,2.3}_fp64"

# Algorithmic FP64 work model of the plain form (FLOPs, an FMA counts 2),
# counted from the kernel source: per quadrature node, per peak Newton
# iteration, per window-end Newton iteration, and a fixed part per Matern
# entry (distance, set-ups, final logs and exp) or per bare K_nu evaluation.
FLOP_NODE, FLOP_PEAK_IT, FLOP_WIN_IT, FLOP_ENTRY_FIXED, FLOP_EVAL_FIXED = 44, 88, 48, 300, 260
# FP64 peak derived from the unit count and clock: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=N_LOC)
    p.add_argument("--cpu-seconds", type=float, default=15.0,
                   help="budget of the CPU oracle baseline sample")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons, "samples": len(rows)}


def kernel_hash():
    h = hashlib.sha256()
    for f in ("bk_plain.cu", "bk_math64.cuh"):
        with open(os.path.join(ROOT, "paper_2502_00356_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(n: int):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, scaled to n^2 output entries; None when the kernel changed since."""
    path = os.path.join(ROOT, "profiles", "matern_sym_f64_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_hash") != kernel_hash():
        return None
    return rec["dram_bytes_per_entry"] * n * n


# ---------------------------------------------------------------------------
def oracle_rate(seconds: float, n: int, threads: int = 0):
    """CPU oracle entries/s on a bounded random sample of the workload."""
    import numpy as np

    import oracle
    from paper_2502_00356_gb300 import inputs
    oracle.build()
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=SEED))
    per_nu = max(1.0, seconds / len(NUS))
    total, elapsed, sizes = 0, 0.0, []
    for k, nu in enumerate(NUS):
        m = 64
        while True:  # grow the sample until it takes a meaningful share of the budget
            I, J = inputs.entry_sample(n, m, seed=300 + k, near_fraction=0.0)
            t0 = time.perf_counter()
            oracle.matern_entries(locs, I, J, SIGMA2, BETA, nu, threads=threads)
            dt = time.perf_counter() - t0
            if dt >= 0.25 * per_nu or m >= 2_000_000:
                break
            m = int(m * min(8.0, max(2.0, 0.3 * per_nu / max(dt, 1e-3))))
        total += m
        elapsed += dt
        sizes.append(m)
    return total / elapsed, sizes, oracle.max_threads() if threads == 0 else threads


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    steps, warm = args.steps, args.warmup
    budget = max(2.0, min(20.0, 150.0 / max(1, steps + warm)))
    for _ in range(warm):
        oracle_rate(min(2.0, budget), args.n)
    rates, sizes = [], None
    t_all = time.perf_counter()
    for _ in range(steps):
        r, sizes, cores = oracle_rate(budget, args.n)
        rates.append(r)
    wall = time.perf_counter() - t_all
    value = statistics.mean(rates)
    per_step_entries = len(NUS) * args.n * args.n
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s",
        "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": 1e3 * per_step_entries / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (long double oracle)",
        "data": "synthetic", "config": config(args.n),
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: random entries of the three matrices "
                                   f"({'/'.join(map(str, sizes))} per nu), "
                                   f"~{budget:.0f} s of CPU work; ms_per_step extrapolates "
                                   f"to the full {len(NUS)} x n^2 entries"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "wall_s": wall,
    }
    print(json.dumps(line), flush=True)


def config(n):
    return {"workload": f"matern_jittered_grid_n{n}_beta{BETA}_nu{{0.5,1.5,2.3}}_fp64",
            "n": n, "sigma2": SIGMA2, "beta": BETA, "nu": list(NUS), "locations": "jittered grid, "
            "Morton order, seed 2", "output_bytes_per_matrix": n * n * 8,
            "l2": "inputs larger than L2: each step writes 3 x n^2 x 8 B of output; no flush",
            "form": "plain FP64 (peak search + eps=2^-52 window + strip-bound node count)",
            "parallelism": "one process per GPU, independent matrices (weak)"}


# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2502_00356_gb300 as bk
    from paper_2502_00356_gb300 import inputs

    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        bk.build()
    if world > 1:
        dist.barrier()
    bk.build()  # no-op when up to date; loads after rank 0 built

    n = args.n
    locs_h = inputs.morton_sorted(inputs.jittered_grid(n, seed=SEED))
    L = torch.as_tensor(locs_h, device=dev)
    out = torch.empty((n, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    # -- work accounting pass (untimed): nodes / iterations per launch
    flop_per_launch = []
    fails = 0
    for nu in NUS:
        ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
        bk.bk_matern_tile(L, SIGMA2, BETA, nu, out=out, opts=bk.make_opts(counters=ctr))
        c = ctr.cpu().numpy()
        fails += int(c[bk.BK_CTR_FAIL])
        flop_per_launch.append(FLOP_NODE * c[bk.BK_CTR_NODES] + FLOP_PEAK_IT * c[bk.BK_CTR_PEAK_ITERS]
                               + FLOP_WIN_IT * c[bk.BK_CTR_ITERS] + FLOP_ENTRY_FIXED * c[bk.BK_CTR_EVALS])
    torch.cuda.synchronize()

    def step(ev=None):
        for k, nu in enumerate(NUS):
            if ev is not None:
                ev[k][0].record(stream)
            bk.bk_matern_tile(L, SIGMA2, BETA, nu, out=out)
            if ev is not None:
                ev[k][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    launch_ms = [[] for _ in NUS]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        evs = []
        for _ in range(args.steps):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in NUS]
            step(ev)
            evs.append(ev)
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    for ev in evs:
        for k in range(len(NUS)):
            launch_ms[k].append(ev[k][0].elapsed_time(ev[k][1]))
    total_ms = t_start.elapsed_time(t_end)
    tmax = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    total_ms = float(tmax.item())
    entries = world * args.steps * len(NUS) * n * n
    value = entries / (total_ms / 1e3)

    # -- roofline of the dominant kernel (the symmetric FP64 tile writer)
    mean_launch_s = statistics.mean(statistics.mean(v) for v in launch_ms) / 1e3
    flop_mean = float(np.mean(flop_per_launch))
    achieved = flop_mean / mean_launch_s / 1e12
    roofline = {"bound": "alu", "kernel": "matern_sym_f64_kernel<double>",
                "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz",
                "traffic": profiled_traffic(n),
                "algorithmic_flop_per_launch": flop_mean,
                "algorithmic_bytes_per_launch": n * n * 8 + 16 * n}

    # -- pipe probes (context for the peak)
    sink = torch.empty(152 * 8 * 256, dtype=torch.float64, device=dev)
    probe = {}
    for kind, name, it in ((0, "fp64_fma_tflops", 2000), (1, "fp32_fma_tflops", 20000),
                           (2, "mufu_ex2_tops", 5000)):
        bk.bk_probe_pipe(kind, it // 10, 152 * 8, 256, sink)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ops = bk.bk_probe_pipe(kind, it, 152 * 8, 256, sink)
        b.record(stream)
        torch.cuda.synchronize()
        mult = 2 if kind in (0, 1) else 1
        probe[name] = ops * mult / (a.elapsed_time(b) / 1e3) / 1e12

    # -- secondary: bare K_nu evaluation, 100,000 pairs (x log-uniform in [1e-3,140], nu in [0.05,10])
    xh, nh = inputs.kv_pairs(100_000, seed=1)
    X, V = torch.as_tensor(xh, device=dev), torch.as_tensor(nh, device=dev)
    Y = torch.empty_like(X)
    for _ in range(3):
        bk.bk_eval(X, V, out=Y)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    reps = 20
    for _ in range(reps):
        bk.bk_eval(X, V, out=Y)
    b.record(stream)
    torch.cuda.synchronize()
    eval_rate = reps * X.numel() / (a.elapsed_time(b) / 1e3)

    # -- end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        locs_pin = torch.from_numpy(locs_h).pin_memory()
        out_pin = torch.empty((n, n), dtype=torch.float64).pin_memory()
        Ld = torch.empty_like(L)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        e_steps = max(1, min(args.steps, 3))
        for _ in range(e_steps):
            for nu in NUS:
                Ld.copy_(locs_pin, non_blocking=True)
                bk.bk_matern_tile(Ld, SIGMA2, BETA, nu, out=out)
                out_pin.copy_(out, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(e_ms, op=dist.ReduceOp.MAX)
        e2e = {"value": world * e_steps * len(NUS) * n * n / (float(e_ms.item()) / 1e3),
               "unit": "entries/s", "h2d_bytes_per_step": len(NUS) * 2 * n * 8,
               "d2h_bytes_per_step": len(NUS) * n * n * 8, "steps": e_steps}
        del out_pin

    cpu = None
    if rank == 0 and world == 1:
        rate, sizes, cores = oracle_rate(args.cpu_seconds, n)
        cpu = {"value": rate, "unit": "entries/s", "cores": cores, "kind": "oracle",
               "sample": f"random entries of the three matrices ({'/'.join(map(str, sizes))} "
                         f"per nu), ~{args.cpu_seconds:.0f} s of CPU work, OpenMP over entries"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(n),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "gpu_launches": args.steps * len(NUS),
            "launch_ms": {str(nu): statistics.mean(v) for nu, v in zip(NUS, launch_ms)},
            "failed_points": fails,
            "eval_fp64": {"value": eval_rate, "unit": "K_nu evals/s",
                          "workload": "100,000 pairs, x log-uniform [1e-3,140], nu U[0.05,10]"},
            "probe": probe,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
