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

# FP64 work model of the plain form in FP64 arithmetic operations (one per
# thread and DFMA/DADD/DMUL): 2 per quadrature node of the common loop (the
# summing FMA and the three-term recurrence of x cosh t; the node's
# exponential, the factor e^{nu t} in its exponent and the geometric factor
# 1 + e^{-2 nu t} run on the integer pipe; windows outside that loop's
# conditions take 9 and are counted at 2), per FP64 peak Newton iteration and
# per FP64 window-end Newton iteration (these run only for windows the check
# rejects, or outside the FP32 search region), and a fixed part per Matern
# entry (the distance, r^2 times the matrix's constant, set-ups, the
# exponent step K nu h, the end terms' scaling, the exponent's FMAs; the
# square root, log x and the final exponential run on the integer pipe).  The
# fixed part is ncu's executed DFMA + DADD + DMUL per evaluation minus 2 x
# nodes per evaluation on the n = 6000 case of the same kernel
# (--profile-case plain_nus: 14.89 for each of nu = 0.5, 1.5, 2.3).
# The FP32 Newton iterations that place the window and the FP32 window check
# run on the FP32/MUFU pipes and are not counted.
OPS_NODE, OPS_PEAK_IT, OPS_WIN_IT, OPS_ENTRY_FIXED = 2, 54, 31, 14.9
# Kernels per bk_matern_tile call of the plain form: the per-launch table of
# e^{-2 nu h} on the quantised steps, then the symmetric tile writer.
LAUNCHES_PER_MATRIX = 2
# FP64 pipe peak from the unit count and clock: 152 SMs x 2 DFMA/clk x 2.07 GHz
# (1.26 TFLOP/s counting an FMA as two FLOPs).
FP64_PEAK_GOPS = 152 * 2 * 2.07e9 / 1e9
# Instruction-issue limit, which bounds the FP32 forms: 152 SMs x 4 warp
# instructions per clock x 32 lanes x 2.07 GHz, in G thread-instructions/s.
ISSUE_PEAK_GINST = 152 * 4 * 32 * 2.07e9 / 1e9


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
    p.add_argument("--no-forms", action="store_true",
                   help="skip the FP32, batched and learned-window measurements")
    p.add_argument("--pairs", type=int, default=100_000_000,
                   help="K_nu pairs of the learned-window evaluation workload")
    p.add_argument("--profile-case", choices=["plain", "plain_nus", "plain_eval", "fp32", "learned",
                                              "learned_eval", "batched", "fp32_forms", "train"],
                   default=None,
                   help="run --warmup launches plus one launch of one kernel on a small case "
                        "(for profiler captures) and exit without a JSON line")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# Multi-rank host logic (weak scaling: each rank builds its own matrices, no
# collective on the data path; the process group only carries the barrier and
# the max over ranks of the timed region).
def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ms: float, world: int, device) -> float:
    """The largest of the ranks' times (every rank calls it; identity at 1)."""
    if world == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, steps: int, units_per_rank_step: float, max_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * steps * units_per_rank_step / (max_ms / 1e3)


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


KERNEL_SOURCES = ("bk_plain.cu", "bk_math64.cuh", "bk_math32.cuh", "bk_forms.cuh", "bk_tiles.cuh",
                  "bk_matern_common.cuh", "bk_exp2_table.inc", "bk_cosh_table.inc")
# The FP32 forms' kernels (single matrix, bare evaluations, batched, learned).
FP32_SOURCES = ("bk_math64.cuh", "bk_math32.cuh", "bk_forms.cuh", "bk_tiles.cuh",
                "bk_matern_common.cuh", "bk_peak_table.inc", "bk_fp32.cu", "bk_learned.cu",
                "bk_batched.cu")


def kernel_hash(files=KERNEL_SOURCES):
    """Hash of the sources a kernel is compiled from (by default the plain
    FP64 tile writer's), with comments removed and whitespace collapsed (so
    that it changes with the compiled code, not with its documentation)."""
    import re
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2502_00356_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profiled_instr():
    """Executed thread instructions per launch of the FP32 forms' bench
    kernels from the committed ncu summary; None when the kernels changed
    since the capture."""
    path = os.path.join(ROOT, "profiles", "fp32_forms_instr.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    return rec if rec.get("kernel_hash") == kernel_hash(FP32_SOURCES) else None


def _traffic_record():
    """The committed ncu record of the dominant kernel, or None when the
    kernel changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "matern_sym_f64_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    return rec if rec.get("kernel_hash") == kernel_hash() else None


def profiled_traffic(n: int):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, scaled to n^2 output entries; None when the kernel changed since."""
    rec = _traffic_record()
    return None if rec is None else rec["dram_bytes_per_entry"] * n * n


def profiled_pipes():
    """Pipe utilisation of the dominant kernel from the committed ncu record
    (--set full on the n = 6000 case): the FP64 pipe, the integer ALU and
    instruction issue, fractions of their peaks; None when the kernel changed."""
    rec = _traffic_record()
    return None if rec is None else rec.get("pipe_utilisation")


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
    rates, sizes, entries = [], None, 0
    t_all = time.perf_counter()
    for _ in range(steps):
        r, sizes, cores = oracle_rate(budget, args.n)
        rates.append(r)
        entries += sum(sizes)
    wall = time.perf_counter() - t_all
    value = statistics.mean(rates)  # each step's rate is timed on its final sample
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "entries/s",
        "n_gpus": world, "steps": steps, "warmup": warm,
        "ms_per_step": 1e3 * wall / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 (long double oracle)",
        "data": "synthetic", "config": config(args.n),
        "entries_per_step": entries / steps,
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle",
                         "sample": f"per step: random entries of the three matrices "
                                   f"({'/'.join(map(str, sizes))} per nu in the last step), "
                                   f"~{budget:.0f} s of CPU work; a step is that bounded "
                                   f"sample, not the full {len(NUS)} x n^2 entries"},
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
def _time(fn, stream, reps=1):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def _max_rel(got, ref, floor=1e-30):
    big = ref.abs() >= floor
    return float(((got.double() - ref.double()).abs() / ref.double().abs().clamp_min(floor))[big].max())


def _counters(bk, dev):
    import torch
    return torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)


def _ctr_summary(bk, c):
    evals = max(1, int(c[bk.BK_CTR_EVALS]))
    return {"evals": int(c[bk.BK_CTR_EVALS]), "nodes_per_eval": float(c[bk.BK_CTR_NODES]) / evals,
            "fallback_rate": float(c[bk.BK_CTR_FALLBACK]) / evals,
            "repairs_per_eval": float(c[bk.BK_CTR_REPAIR]) / evals,
            "newton_iters_per_eval": float(c[bk.BK_CTR_ITERS] + c[bk.BK_CTR_PEAK_ITERS]) / evals,
            "failed": int(c[bk.BK_CTR_FAIL])}


def issue_roofline(key, kernel, launch_s, evals):
    """Roofline of an FP32-form kernel, which is bound by instruction issue:
    achieved = the kernel's executed thread instructions per launch (ncu,
    profiles/fp32_forms_instr.json, same workload, null when the kernels
    changed since the capture) / the live CUDA-event launch time, against the
    issue limit 152 SMs x 4 warp instructions/clk x 32 lanes x 2.07 GHz.
    Divergence (inactive lanes) and issue stalls both lower it."""
    rec = profiled_instr()
    d = (rec or {}).get("kernels", {}).get(key)
    achieved = d["thread_inst"] / launch_s / 1e9 if d else None
    out = {"bound": "alu", "kernel": kernel, "unit": "G thread-instr/s",
           "peak": ISSUE_PEAK_GINST, "peak_source": "derived: 152 SMs x 4 warp-instr/clk x 32 "
           "lanes x 2.07 GHz (of derived)", "achieved": achieved,
           "frac": achieved / ISSUE_PEAK_GINST if achieved else None,
           "launch_ms": 1e3 * launch_s, "evals_per_launch": evals}
    if d:
        out["thread_inst_per_eval"] = d["thread_inst"] / max(1, evals)
        out["lanes_active_of_32"] = d["thread_inst"] / d["warp_inst"]
    return out


def measure_forms(bk, inputs, dev, stream, args, plain_rate):
    """Throughput, roofline, counters and output samples of the other forms
    (outside the headline timing).  The samples are checked against the
    oracle by the CPU leg (oracle_checks)."""
    import numpy as np
    import torch

    res, samples = {}, []
    net = bk.LearnedWindow(path=os.path.join(ROOT, "paper_2502_00356_gb300", "weights",
                                             "window_mlp.bkw"))

    def sample_matrix(key, out, locs_h, sigma2, beta, nu, m, seed, near):
        n = locs_h.shape[1]
        I, J = inputs.entry_sample(n, m, seed=seed, near_fraction=near)
        got = out[torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)]  # (i, j) at out[j, i]
        samples.append({"key": key, "kind": "matern", "locs": locs_h, "I": I, "J": J,
                        "theta": (sigma2, beta, nu), "got": got.double().cpu().numpy()})

    # -- C3, FP32 precision form: n = 40,000 jittered grid (seed 4), beta = 0.05,
    # nu ~ U(0.3, 3.5) (seed 5), FP32 out; error on a seeded 10^6-entry sample (seed 6,
    # 1 % nearest-neighbour pairs)
    n3, beta3 = 40_000, 0.05
    nu3 = float(np.random.default_rng(5).uniform(0.3, 3.5))
    L3h = inputs.morton_sorted(inputs.jittered_grid(n3, seed=4))
    L3 = torch.as_tensor(L3h, device=dev)
    o32 = torch.empty((n3, n3), dtype=torch.float32, device=dev)
    c = _counters(bk, dev)
    bk.bk_matern_tile(L3, 1.0, beta3, nu3, out=o32, opts=bk.make_opts(compute=bk.BK_F32, counters=c))
    cs = _ctr_summary(bk, c.cpu().numpy())
    t = _time(lambda: bk.bk_matern_tile(L3, 1.0, beta3, nu3, out=o32), stream, 3)
    res["fp32_matern"] = {
        "workload": f"C3: n={n3} jittered grid, beta={beta3}, nu={nu3:.4f} (U(0.3,3.5), seed 5), "
                    "FP32 out", "value": n3 * n3 / t, "unit": "entries/s", "ms": 1e3 * t,
        "counters": cs, "roofline": issue_roofline("fp32_matern", "matern_sym_kernel<FormF32, float>",
                                                   t, cs["evals"])}
    sample_matrix("fp32_matern", o32, L3h, 1.0, beta3, nu3, 1_000_000, 6, 0.01)

    # -- C5 matrix: learned window vs searched window vs plain FP64, n = 40,000, beta = 0.1,
    # nu = 1.7, FP32 out; error on a 10^5-entry sample (seed 7)
    n5, beta5, nu5 = 40_000, 0.1, 1.7
    c_l = _counters(bk, dev)
    o_l = o32
    bk.bk_matern_tile(L3, 1.0, beta5, nu5, out=o_l, opts=bk.make_opts(learned=net, counters=c_l))
    cl = _ctr_summary(bk, c_l.cpu().numpy())
    lo = bk.make_opts(learned=net)
    t_l = _time(lambda: bk.bk_matern_tile(L3, 1.0, beta5, nu5, out=o_l, opts=lo), stream, 3)
    sample_matrix("learned_matern", o_l, L3h, 1.0, beta5, nu5, 100_000, 7, 0.01)
    t_s = _time(lambda: bk.bk_matern_tile(L3, 1.0, beta5, nu5, out=o_l), stream, 3)
    del o32, o_l
    torch.cuda.empty_cache()
    o64 = torch.empty((n5, n5), dtype=torch.float64, device=dev)
    t_p = _time(lambda: bk.bk_matern_tile(L3, 1.0, beta5, nu5, out=o64), stream, 1)
    del o64
    torch.cuda.empty_cache()
    res["learned_matern"] = {
        "workload": f"C5: n={n5} jittered grid, beta={beta5}, nu={nu5}, FP32 out",
        "value": n5 * n5 / t_l, "fp32_search_value": n5 * n5 / t_s,
        "plain_fp64_value": n5 * n5 / t_p, "unit": "entries/s",
        "learned_over_plain": t_p / t_l, "learned_over_fp32_search": t_s / t_l,
        "counters": cl, "fallback_rate": cl["fallback_rate"],
        "roofline": issue_roofline("learned_matern", "matern_sym_kernel<FormF32Learned, float>",
                                   t_l, cl["evals"])}
    del L3
    torch.cuda.empty_cache()

    # -- C5 evaluations: 10^8 pairs, x log-uniform [1e-3, 140], nu U[0.05, 20] (seed 8), FP32
    # out; lanes per evaluation chosen by bk_eval_autotune; error on 10^6 of the pairs (seed 9)
    npairs = args.pairs
    xh, nh = inputs.kv_pairs(npairs, seed=8, nu_lo=0.05, nu_hi=20.0)
    X, V = torch.as_tensor(xh, device=dev), torch.as_tensor(nh, device=dev)
    Y = torch.empty(npairs, dtype=torch.float32, device=dev)
    lanes_l = bk.bk_eval_autotune(X, V, Y, lo)
    fo = bk.make_opts(compute=bk.BK_F32)
    lanes_f = bk.bk_eval_autotune(X, V, Y, fo)
    c_e = _counters(bk, dev)
    bk.bk_eval_ex(X, V, out=Y, opts=bk.make_opts(learned=net, counters=c_e))
    ce = _ctr_summary(bk, c_e.cpu().numpy())
    t_le = _time(lambda: bk.bk_eval_ex(X, V, out=Y, opts=lo), stream, 3)
    per_lanes = {}
    for L in (1, 2, 4, 8):
        oL = bk.make_opts(learned=net, lanes=L)
        per_lanes[str(L)] = npairs / _time(lambda: bk.bk_eval_ex(X, V, out=Y, opts=oL), stream, 2)
    bk.bk_eval_ex(X, V, out=Y, opts=lo)
    idx = np.sort(np.random.default_rng(9).choice(npairs, 1_000_000, replace=False))
    got_l = Y[torch.as_tensor(idx, device=dev)].double().cpu().numpy()
    samples.append({"key": "learned_eval", "kind": "eval", "x": xh[idx], "nu": nh[idx], "got": got_l})
    c_f = _counters(bk, dev)
    bk.bk_eval_ex(X, V, out=Y, opts=bk.make_opts(compute=bk.BK_F32, counters=c_f))
    cf = _ctr_summary(bk, c_f.cpu().numpy())
    t_se = _time(lambda: bk.bk_eval_ex(X, V, out=Y, opts=fo), stream, 3)
    sub = slice(0, 2_000_000)
    Yd = torch.empty(2_000_000, dtype=torch.float64, device=dev)
    t_pe = _time(lambda: bk.bk_eval(X[sub], V[sub], out=Yd), stream, 1)
    res["learned_eval"] = {
        "workload": f"C5: {npairs} pairs, x log-uniform [1e-3,140], nu U[0.05,20] (seed 8), FP32 out",
        "value": npairs / t_le, "unit": "K_nu evals/s", "lanes": lanes_l,
        "value_per_lanes": per_lanes, "fp32_search_value": npairs / t_se,
        "fp32_search_lanes": lanes_f, "plain_fp64_value": 2_000_000 / t_pe,
        "counters": ce, "fallback_rate": ce["fallback_rate"], "fp32_search_counters": cf,
        "roofline": issue_roofline("learned_eval" if lanes_l == 1 else f"learned_eval_L{lanes_l}",
                                   f"eval_coop_kernel<FormF32Learned, float, {lanes_l}>",
                                   t_le, ce["evals"]),
        "fp32_search_roofline": issue_roofline("fp32_eval" if lanes_f == 1 else f"fp32_eval_L{lanes_f}",
                                               f"eval_coop_kernel<FormF32, float, {lanes_f}>",
                                               t_se, cf["evals"])}
    del X, V, Y, Yd
    torch.cuda.empty_cache()

    # -- C4 batched sweep: 256 instances, n log-uniform [500, 8000], one persistent launch
    # replayed from a CUDA graph; the learned FP32 output sampled (400 entries per instance)
    insts = inputs.batched_instances(256)
    entries = sum(i.n * i.n for i in insts)
    locs_h = [i.locations() for i in insts]
    locs = [torch.as_tensor(h, device=dev) for h in locs_h]
    bres = {"workload": "C4: 256 instances, n log-uniform [500, 8000], sigma2 U[0.5,2], "
                        "beta U[0.02,0.3], nu U[0.3,3], one launch replayed from a CUDA graph",
            "entries": entries}
    for name, dtype, form_opts in (("fp64", torch.float64, {}),
                                   ("fp32", torch.float32, {}),
                                   ("learned_fp32", torch.float32, {"learned": net})):
        outs = [torch.empty((i.n, i.n), dtype=dtype, device=dev) for i in insts]
        d = bk.make_descs([(L, i.sigma2, i.beta, i.nu, o) for L, i, o in zip(locs, insts, outs)])
        cb = _counters(bk, dev)
        cplan = bk.BatchedPlan([i.n for i in insts], dtype=dtype,
                               opts=bk.make_opts(counters=cb, **form_opts) if form_opts else
                               bk.make_opts(compute=bk.BK_F64 if dtype == torch.float64 else bk.BK_F32,
                                            counters=cb))
        bk.bk_matern_batched(d, cplan)
        cbs = _ctr_summary(bk, cb.cpu().numpy())
        del cplan
        plan = bk.BatchedPlan([i.n for i in insts], dtype=dtype,
                              opts=bk.make_opts(**form_opts) if form_opts else None)
        plan.autotune(d, sample_tiles=20_000)
        bk.bk_matern_batched(d, plan)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            bk.bk_matern_batched(d, plan)
        tb = _time(g.replay, stream, 2 if name == "fp64" else 5)
        bres[name] = {"value": entries / tb, "unit": "entries/s", "ms": 1e3 * tb,
                      "plan": plan.info(), "counters": cbs}
        if not form_opts:  # the allocation-free entry point on the same sweep (no plan)
            bk.bk_matern_batched_static(d, len(insts), dtype=dtype)
            ts = _time(lambda: bk.bk_matern_batched_static(d, len(insts), dtype=dtype), stream,
                       2 if name == "fp64" else 5)
            bres[name]["static_value"] = entries / ts
        if name != "fp64":
            key = "batched_" + name
            kern = ("matern_batched_kernel<FormF32Learned, float>" if form_opts
                    else "matern_batched_kernel<FormF32, float>")
            bres[name]["roofline"] = issue_roofline(key, kern, tb, cbs["evals"])
        if name == "learned_fp32":
            bres[name]["fallback_rate"] = cbs["fallback_rate"]
            for k, (inst, o) in enumerate(zip(insts, outs)):
                I, J = inputs.entry_sample(inst.n, 400, seed=1000 + k, near_fraction=0.01)
                got = o[torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)]
                samples.append({"key": "batched_learned_fp32", "kind": "matern", "locs": locs_h[k],
                                "I": I, "J": J, "theta": (inst.sigma2, inst.beta, inst.nu),
                                "got": got.double().cpu().numpy()})
        del outs, d, g, plan
        torch.cuda.empty_cache()
    bres["learned_fp32_over_fp64"] = bres["learned_fp32"]["value"] / bres["fp64"]["value"]
    res["batched"] = bres
    res["learned_batched_over_plain_fp64_headline"] = bres["learned_fp32"]["value"] / plain_rate
    del locs
    torch.cuda.empty_cache()

    # -- the paper's refined algorithm (Algorithm 2: Temme's series below x = 0.1, the fixed
    # window [0, 9] with b bins above) on the headline matrices, b in {16, 40, 128}
    L2 = torch.as_tensor(inputs.morton_sorted(inputs.jittered_grid(N_LOC, seed=SEED)), device=dev)
    o2 = torch.empty((N_LOC, N_LOC), dtype=torch.float64, device=dev)
    cols2 = slice(0, 1000)
    alg = {"workload": f"n={N_LOC} jittered grid, beta={BETA}, nu in {list(NUS)}, FP64 out "
                       "(the headline matrices)",
           "unit": "entries/s",
           "err": "max |entry - plain FP64 form| over the first 1000 columns (entries <= 1)"}
    refs = {nu: bk.bk_matern_tile2(L2, L2[:, cols2].contiguous(), SIGMA2, BETA, nu) for nu in NUS}
    for bins in (16, 40, 128):
        ts, errs = [], []
        for nu in NUS:
            op = bk.paper_algorithm2_opts(bins=bins)
            bk.bk_matern_tile(L2, SIGMA2, BETA, nu, out=o2, opts=op)
            ts.append(_time(lambda: bk.bk_matern_tile(L2, SIGMA2, BETA, nu, out=o2, opts=op),
                            stream, 1))
            errs.append(float((o2[cols2, :] - refs[nu]).abs().max()))
        alg[f"b{bins}"] = {"value": len(NUS) * N_LOC * N_LOC / sum(ts),
                           "launch_ms": [1e3 * t for t in ts], "max_abs_err": max(errs),
                           "plain_form_speedup": plain_rate * sum(ts) / (len(NUS) * N_LOC * N_LOC)}
    res["paper_algorithm2"] = alg
    del o2, L2, refs
    torch.cuda.empty_cache()

    # -- downstream Gaussian log-likelihood (blocked FP64 Cholesky) on the n = 4,000 and
    # n = 8,000 Matern matrices of the Cholesky checks (jittered grid seed 3, beta 0.1, nu 0.5)
    ll = {"unit": "s", "workload": "jittered grid (seed 3), sigma2 1, beta 0.1, nu 0.5, "
                                   "z ~ N(0, 1) (seed 5): matrix generation + log-likelihood"}
    for nl in (4000, 8000):
        Ll = torch.as_tensor(inputs.morton_sorted(inputs.jittered_grid(nl, seed=3)), device=dev)
        zl = torch.as_tensor(np.random.default_rng(5).standard_normal(nl), device=dev)
        ml = torch.empty((nl, nl), dtype=torch.float64, device=dev)
        yl = torch.empty(nl, dtype=torch.float64, device=dev)
        outl = torch.empty(3, dtype=torch.float64, device=dev)
        bk.bk_matern_tile(Ll, SIGMA2, BETA, 0.5, out=ml)
        bk.bk_gaussian_loglik(ml, zl, y=yl, out=outl)
        t_gen = _time(lambda: bk.bk_matern_tile(Ll, SIGMA2, BETA, 0.5, out=ml), stream, 1)
        t_ll = _time(lambda: bk.bk_gaussian_loglik(ml, zl, y=yl, out=outl), stream, 1)
        bk.bk_matern_tile(Ll, SIGMA2, BETA, 0.5, out=ml)  # the last call factored ml in place
        ll[f"n{nl}"] = {"matern_s": t_gen, "loglik_s": t_ll,
                        "cholesky_fp64_tflops": nl ** 3 / 3 / t_ll / 1e12,
                        "loglik": float(bk.bk_gaussian_loglik(ml, zl, y=yl, out=outl)[0])}
        del Ll, zl, ml, yl
        torch.cuda.empty_cache()
    res["gaussian_loglik"] = ll
    return res, samples


def oracle_checks(samples, headline_samples):
    """The CPU leg's comparison of GPU output samples with the oracle (OpenMP
    over all host cores): the FP32 forms against the oracle's FP64 instance
    (1e-5 tolerances), the plain FP64 headline against the long double oracle
    (1e-10 absolute).  Returns {key: {...}} and the seconds spent."""
    import numpy as np

    import oracle
    oracle.build()
    t0 = time.perf_counter()
    out = {}
    groups = {}
    for smp in samples:
        groups.setdefault(smp["key"], []).append(smp)
    for key, lst in groups.items():
        worst, m = 0.0, 0
        for smp in lst:
            if smp["kind"] == "eval":
                ref = oracle.besselk_f64(smp["x"], smp["nu"])
            else:
                ref = oracle.matern_entries_f64(smp["locs"], smp["I"], smp["J"], *smp["theta"])
            got = smp["got"]
            ok = (np.abs(ref) >= 1e-30) & (np.abs(ref) < 3.0e38)  # FP32-representable entries
            rel = np.abs(got[ok] / ref[ok] - 1.0)
            worst = max(worst, float(rel.max()) if rel.size else 0.0)
            m += got.size
        out[key] = {"max_rel_vs_oracle": worst, "sample": m, "oracle": "FP64 instance"}
    for nu, (locs, I, J, got) in headline_samples.items():
        ref = oracle.matern_entries(locs, I, J, SIGMA2, BETA, nu)
        out.setdefault("plain_fp64", {"max_abs_vs_oracle": 0.0, "sample": 0,
                                      "oracle": "long double"})
        d = out["plain_fp64"]
        d["max_abs_vs_oracle"] = max(d["max_abs_vs_oracle"], float(np.abs(got - ref).max()))
        d["sample"] += got.size
    return out, time.perf_counter() - t0


def measure_e2e(bk, locs_h, n, dev, stream, args, world, device_step_ms):
    """The headline metric through bk_matern_tile_host: per step the three
    matrices, each from host locations to a pinned host matrix (transfers in
    the timed region; the tile writer stores into the host matrix directly).
    Also reports the copy-engine bandwidth of one matrix (device -> pinned
    host and back) and the share of that copy time the direct stores hide."""
    import torch
    locs_pin = torch.from_numpy(locs_h).pin_memory()
    outs = [torch.empty((n, n), dtype=torch.float64, pin_memory=True) for _ in NUS]
    work = torch.empty(bk.matern_tile_host_workspace(n, staged=True), dtype=torch.uint8,
                       device=dev)

    def step(staged=False):
        for o, nu in zip(outs, NUS):
            bk.bk_matern_tile_host(locs_pin, SIGMA2, BETA, nu, o, work, staged=staged,
                                   stream=stream)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    e_ms = max_over_ranks(a.elapsed_time(b), world, dev)
    # the staged way (matrix in the workspace, finished panels copied out), timed
    # the same way, for comparison
    step(staged=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(max(1, args.steps // 2)):
        step(staged=True)
    b.record(stream)
    torch.cuda.synchronize()
    staged_ms = a.elapsed_time(b) / max(1, args.steps // 2)
    # plain copies of one matrix, device -> pinned host and back (bandwidth)
    mat = work[-n * n * 8:].view(torch.float64)
    d2h = _time(lambda: outs[0].view(-1).copy_(mat, non_blocking=True), stream, 3)
    h2d = _time(lambda: mat.copy_(outs[0].view(-1), non_blocking=True), stream, 3)
    copy_ms = len(NUS) * d2h * 1e3
    step_ms = e_ms / args.steps
    hidden = 1.0 - max(0.0, step_ms - device_step_ms) / copy_ms
    ok = all(bool(torch.isfinite(o[:: max(1, n // 97), :: max(1, n // 89)]).all()) for o in outs)
    del outs, work
    torch.cuda.empty_cache()
    return {"value": job_rate(world, args.steps, len(NUS) * n * n, e_ms), "unit": "entries/s",
            "h2d_bytes_per_step": len(NUS) * 2 * n * 8,
            "d2h_bytes_per_step": len(NUS) * n * n * 8, "steps": args.steps,
            "warmup": max(1, args.warmup), "ms_per_step": step_ms,
            "call": "bk_matern_tile_host (host locations in; the kernel stores into the "
                    "pinned host matrix)",
            "d2h_gbs": n * n * 8 / d2h / 1e9, "h2d_gbs": n * n * 8 / h2d / 1e9,
            "copy_hidden_fraction": hidden, "device_only_ms_per_step": device_step_ms,
            "staged_value": len(NUS) * n * n / (staged_ms / 1e3),
            "host_output_finite": ok}


def profile_case(args):
    """Small single-kernel cases whose outputs still exceed the 129 MB L2."""
    import numpy as np
    import torch

    import paper_2502_00356_gb300 as bk
    from paper_2502_00356_gb300 import inputs
    bk.build()
    dev = torch.device("cuda")
    c = args.profile_case
    if c == "fp32_forms":
        return profile_fp32_forms(args, bk, inputs, dev)
    if c == "plain_nus":
        return profile_plain_nus(bk, inputs, dev)
    if c == "train":
        return profile_train(args, bk, dev)
    net = None
    if c in ("learned", "learned_eval", "batched"):
        net = bk.LearnedWindow(path=os.path.join(ROOT, "paper_2502_00356_gb300", "weights",
                                                 "window_mlp.bkw"))
    if c in ("plain", "fp32", "learned"):
        n = {"plain": 6000, "fp32": 12000, "learned": 12000}[c]
        L = torch.as_tensor(inputs.morton_sorted(inputs.jittered_grid(n, seed=4)), device=dev)
        dtype = torch.float64 if c == "plain" else torch.float32
        out = torch.empty((n, n), dtype=dtype, device=dev)
        beta, nu = (0.1, 0.5) if c == "plain" else ((0.05, 2.876) if c == "fp32" else (0.1, 1.7))
        opts = bk.make_opts(learned=net) if c == "learned" else None
        run = lambda: bk.bk_matern_tile(L, 1.0, beta, nu, out=out, opts=opts)
    elif c == "plain_eval":
        # the plain FP64 bare evaluation on 10^7 pairs of the 100,000-pair
        # workload's distribution (x log-uniform in [1e-3, 140], nu in [0.05,
        # 10]): 240 MB of inputs and output, above the L2
        xh, nh = inputs.kv_pairs(10_000_000, seed=1)
        X, V = torch.as_tensor(xh, device=dev), torch.as_tensor(nh, device=dev)
        Y = torch.empty(X.numel(), dtype=torch.float64, device=dev)
        run = lambda: bk.bk_eval(X, V, out=Y)
    elif c == "learned_eval":
        xh, nh = inputs.kv_pairs(20_000_000, seed=8, nu_lo=0.05, nu_hi=20.0)
        X, V = torch.as_tensor(xh, device=dev), torch.as_tensor(nh, device=dev)
        Y = torch.empty(X.numel(), dtype=torch.float32, device=dev)
        opts = bk.make_opts(learned=net)
        run = lambda: bk.bk_eval_ex(X, V, out=Y, opts=opts)
    else:
        insts = inputs.batched_instances(32)
        locs = [torch.as_tensor(i.locations(), device=dev) for i in insts]
        outs = [torch.empty((i.n, i.n), dtype=torch.float32, device=dev) for i in insts]
        d = bk.make_descs([(L, i.sigma2, i.beta, i.nu, o) for L, i, o in zip(locs, insts, outs)])
        plan = bk.BatchedPlan([i.n for i in insts], dtype=torch.float32)
        run = lambda: bk.bk_matern_batched(d, plan)
    for _ in range(args.warmup + 1):
        run()
    torch.cuda.synchronize()


def profile_plain_nus(bk, inputs, dev):
    """The plain FP64 tile writer on the n = 6,000 case for nu = 0.5, 1.5 and
    2.3: one launch each with the counters (nodes per entry, printed as one
    JSON line), then one launch each without them, the three launches an FP64
    instruction-count capture takes (-k regex:matern_sym -s 3 -c 3)."""
    import torch
    n = 6000
    L = torch.as_tensor(inputs.morton_sorted(inputs.jittered_grid(n, seed=4)), device=dev)
    out = torch.empty((n, n), dtype=torch.float64, device=dev)
    res = {}
    for nu in NUS:
        c = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
        bk.bk_matern_tile(L, 1.0, BETA, nu, out=out, opts=bk.make_opts(counters=c))
        c = c.cpu().numpy()
        res[str(nu)] = {"entries": n * n, "evals": int(c[bk.BK_CTR_EVALS]),
                        "nodes_per_eval": float(c[bk.BK_CTR_NODES]) / max(1, int(c[bk.BK_CTR_EVALS])),
                        "fallback": int(c[bk.BK_CTR_FALLBACK])}
    for nu in NUS:
        bk.bk_matern_tile(L, 1.0, BETA, nu, out=out)
    torch.cuda.synchronize()
    print(json.dumps(res))


def profile_train(args, bk, dev):
    """Window-network training steps of batch 8,192 on synthetic labelled
    points (2^20): --warmup + 1 steps of the tensor-core step kernel
    (mlp_train_tc_kernel), then as many of the FP32 SIMT one; the mean time
    per step of each over 200 more is printed as one JSON line."""
    import numpy as np
    import torch
    rng = np.random.default_rng(1)
    n = 1 << 20
    x = np.exp(rng.uniform(math.log(1e-3), math.log(140.0), n))
    nu = rng.uniform(0.05, 20.0, n)
    ts = rng.uniform(0.0, 8.0, n)
    lab = np.stack([ts, np.maximum(ts - rng.uniform(0.5, 4.0, n), 0.0), ts + rng.uniform(0.5, 4.0, n),
                    -x, rng.uniform(5.0, 40.0, n), np.zeros(n)], axis=1)
    X, V, Lb = (torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in (x, nu, lab))
    res = {}
    for path, name in ((bk.BK_TRAIN_TENSOR, "tensor"), (bk.BK_TRAIN_SIMT, "simt")):
        net = bk.LearnedWindow(seed=1)
        net.set_train_path(path)
        net.train(X, V, Lb, steps=args.warmup + 1, batch=8192)
        torch.cuda.synchronize()
        res[name + "_us_per_step"] = round(1e6 * _time(
            lambda: net.train(X, V, Lb, steps=200, batch=8192), torch.cuda.current_stream()) / 200, 2)
        net.params()  # raises if a tensor-core step gave up waiting
    print(json.dumps(res))


def profile_fp32_forms(args, bk, inputs, dev):
    """One launch of each FP32-form kernel the bench times, on the bench's own
    workloads, in this order: the C3 FP32 matrix, the C5 learned matrix, the
    10^8 learned and FP32 bare evaluations (1 lane per evaluation), and the
    C4 batched FP32 and learned sweeps (for a one-pass ncu instruction count;
    --warmup W runs each W more times first)."""
    import numpy as np
    import torch
    net = bk.LearnedWindow(path=os.path.join(ROOT, "paper_2502_00356_gb300", "weights",
                                             "window_mlp.bkw"))
    L3 = torch.as_tensor(inputs.morton_sorted(inputs.jittered_grid(40_000, seed=4)), device=dev)
    o = torch.empty((40_000, 40_000), dtype=torch.float32, device=dev)
    nu3 = float(np.random.default_rng(5).uniform(0.3, 3.5))
    lo = bk.make_opts(learned=net)
    runs = [lambda: bk.bk_matern_tile(L3, 1.0, 0.05, nu3, out=o),
            lambda: bk.bk_matern_tile(L3, 1.0, 0.1, 1.7, out=o, opts=lo)]
    for r in runs:
        for _ in range(args.warmup + 1):
            r()
    torch.cuda.synchronize()
    del o, L3
    torch.cuda.empty_cache()
    xh, nh = inputs.kv_pairs(args.pairs, seed=8, nu_lo=0.05, nu_hi=20.0)
    X, V = torch.as_tensor(xh, device=dev), torch.as_tensor(nh, device=dev)
    Y = torch.empty(args.pairs, dtype=torch.float32, device=dev)
    for opts in (bk.make_opts(learned=net, lanes=1), bk.make_opts(compute=bk.BK_F32, lanes=1)):
        for _ in range(args.warmup + 1):
            bk.bk_eval_ex(X, V, out=Y, opts=opts)
    torch.cuda.synchronize()
    del X, V, Y
    torch.cuda.empty_cache()
    insts = inputs.batched_instances(256)
    locs = [torch.as_tensor(i.locations(), device=dev) for i in insts]
    for opts in (None, lo):
        outs = [torch.empty((i.n, i.n), dtype=torch.float32, device=dev) for i in insts]
        d = bk.make_descs([(L, i.sigma2, i.beta, i.nu, o) for L, i, o in zip(locs, insts, outs)])
        plan = bk.BatchedPlan([i.n for i in insts], dtype=torch.float32, opts=opts)
        for _ in range(args.warmup + 1):
            bk.bk_matern_batched(d, plan)
        torch.cuda.synchronize()
        del outs, d, plan
        torch.cuda.empty_cache()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_case is not None:
        profile_case(args)
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
    barrier(world)
    bk.build()  # no-op when up to date; loads after rank 0 built

    n = args.n
    locs_h = inputs.morton_sorted(inputs.jittered_grid(n, seed=SEED))
    L = torch.as_tensor(locs_h, device=dev)
    out = torch.empty((n, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    # -- work accounting pass (untimed): nodes / iterations per launch
    flop_per_launch = []
    work = []
    fails = fallbacks = evals_counted = 0
    for nu in NUS:
        ctr = torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)
        bk.bk_matern_tile(L, SIGMA2, BETA, nu, out=out, opts=bk.make_opts(counters=ctr))
        c = ctr.cpu().numpy()
        fails += int(c[bk.BK_CTR_FAIL])
        fallbacks += int(c[bk.BK_CTR_FALLBACK])
        evals_counted += int(c[bk.BK_CTR_EVALS])
        work.append({"nu": nu, "nodes_per_entry": float(c[bk.BK_CTR_NODES] / max(1, c[bk.BK_CTR_EVALS])),
                     "iters_per_entry": float(c[bk.BK_CTR_ITERS] / max(1, c[bk.BK_CTR_EVALS])),
                     "peak_iters_per_entry": float(c[bk.BK_CTR_PEAK_ITERS]
                                                   / max(1, c[bk.BK_CTR_EVALS]))})
        flop_per_launch.append(OPS_NODE * c[bk.BK_CTR_NODES] + OPS_PEAK_IT * c[bk.BK_CTR_PEAK_ITERS]
                               + OPS_WIN_IT * c[bk.BK_CTR_ITERS] + OPS_ENTRY_FIXED * c[bk.BK_CTR_EVALS])
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
    barrier(world)
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
    barrier(world)
    for ev in evs:
        for k in range(len(NUS)):
            launch_ms[k].append(ev[k][0].elapsed_time(ev[k][1]))
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world, dev)
    value = job_rate(world, args.steps, len(NUS) * n * n, total_ms)

    # -- output samples of the headline matrices for the CPU leg's oracle check
    # (10^4 seeded entries per nu, 1 % nearest-neighbour pairs; untimed)
    headline_samples = {}
    for k, nu in enumerate(NUS):
        bk.bk_matern_tile(L, SIGMA2, BETA, nu, out=out)
        I, J = inputs.entry_sample(n, 10_000, seed=400 + k, near_fraction=0.01)
        got = out[torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)].cpu().numpy()
        headline_samples[nu] = (locs_h, I, J, got)

    # -- roofline of the dominant kernel (the symmetric FP64 tile writer)
    mean_launch_s = statistics.mean(statistics.mean(v) for v in launch_ms) / 1e3
    flop_mean = float(np.mean(flop_per_launch))
    achieved = flop_mean / mean_launch_s / 1e9
    roofline = {"bound": "alu", "kernel": "matern_sym_kernel<FormF64T<false>, double>",
                "achieved": achieved, "peak": FP64_PEAK_GOPS, "unit": "FP64 Gop/s",
                "frac": achieved / FP64_PEAK_GOPS,
                "peak_source": "derived: 152 SMs x 2 FP64 ops/clk x 2.07 GHz (of derived)",
                "traffic": profiled_traffic(n),
                "pipes_ncu": profiled_pipes(),
                "algorithmic_fp64_ops_per_launch": flop_mean,
                "algorithmic_bytes_per_launch": n * n * 8 + 16 * n,
                "work": work}

    # -- pipe probes (context for the peak)
    sink = torch.empty(152 * 8 * 256, dtype=torch.float64, device=dev)
    probe = {}
    for kind, name, it in ((0, "fp64_fma_tflops", 2000), (1, "fp32_fma_tflops", 20000),
                           (2, "mufu_ex2_tops", 5000), (3, "cvt_f64_to_f32_tops", 2000),
                           (4, "cvt_f32_to_f64_tops", 2000)):
        bk.bk_probe_pipe(kind, it // 10, 152 * 8, 256, sink)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ops = bk.bk_probe_pipe(kind, it, 152 * 8, 256, sink)
        b.record(stream)
        torch.cuda.synchronize()
        mult = 2 if kind in (0, 1) else 1  # an FMA counts 2 FLOPs
        probe[name] = ops * mult / (a.elapsed_time(b) / 1e3) / 1e12
    # Measured context for the derived peaks: the DFMA probe's operations/s (a
    # stream of independent FP64 FMAs reaches ~0.8 of the unit-count rate,
    # below the FP64 operations/s the tile writer itself sustains, so it is no
    # ceiling), and the FFMA probe's thread instructions/s (the issue limit).
    dfma_gops = probe["fp64_fma_tflops"] / 2 * 1e3
    issue_ginst = probe["fp32_fma_tflops"] / 2 * 1e3
    roofline.update({"peak_measured": dfma_gops, "frac_measured": achieved / dfma_gops,
                     "peak_measured_source": "bk_probe_pipe kind 0 (independent DFMA chains)"})

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
    # K with dK/dx and dK/dnu from one quadrature, same pairs
    G = [torch.empty_like(X) for _ in range(3)]
    bk.bk_eval_grad(X, V, *G)
    a.record(stream)
    for _ in range(reps):
        bk.bk_eval_grad(X, V, *G)
    b.record(stream)
    torch.cuda.synchronize()
    grad_rate = reps * X.numel() / (a.elapsed_time(b) / 1e3)
    del G

    # -- end to end through the C-ABI with HOST buffers: bk_matern_tile_host takes
    # the locations from pinned host memory and the tile writer stores each matrix
    # straight into a pinned host matrix over NVLink-C2C.
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(bk, locs_h, n, dev, stream, args, world, total_ms / args.steps)

    forms, samples = None, []
    if not args.no_forms:
        del out
        torch.cuda.empty_cache()
        forms, samples = measure_forms(bk, inputs, dev, stream, args, value)

    if forms is not None:
        for r in ([forms["fp32_matern"]["roofline"], forms["learned_matern"]["roofline"],
                   forms["learned_eval"]["roofline"], forms["learned_eval"]["fp32_search_roofline"]]
                  + [forms["batched"][k]["roofline"] for k in ("fp32", "learned_fp32")]):
            r["peak_measured"] = issue_ginst
            r["peak_measured_source"] = "bk_probe_pipe kind 1 (independent FFMA chains)"
            r["frac_measured"] = r["achieved"] / issue_ginst if r["achieved"] else None

    # -- the CPU leg (rank 0 at N = 1): the oracle timed on a bounded sample of the
    # workload, and the oracle's values for the GPU output samples (errors)
    cpu, checks = None, None
    if rank == 0 and world == 1:
        rate, sizes, cores = oracle_rate(args.cpu_seconds, n)
        cpu = {"value": rate, "unit": "entries/s", "cores": cores, "kind": "oracle",
               "sample": f"random entries of the three matrices ({'/'.join(map(str, sizes))} "
                         f"per nu), ~{args.cpu_seconds:.0f} s of CPU work, OpenMP over entries"}
        checks, check_s = oracle_checks(samples, headline_samples)
        cpu["error_checks_s"] = check_s
        if forms is not None:
            for key, d in checks.items():
                if key == "batched_learned_fp32":
                    forms["batched"]["learned_fp32"].update(d)
                elif key in forms:
                    forms[key].update(d)
                elif key == "fp32_eval":
                    forms["learned_eval"]["fp32_search_error"] = d

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "entries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config(n),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "clocks": clk.summary(), "gpu_launches": args.steps * len(NUS) * LAUNCHES_PER_MATRIX,
            "launch_ms": {str(nu): statistics.mean(v) for nu, v in zip(NUS, launch_ms)},
            "failed_points": fails,
            "error_vs_oracle": (checks or {}).get("plain_fp64"),
            "plain_window_fallback_rate": fallbacks / max(evals_counted, 1),
            "eval_fp64": {"value": eval_rate, "unit": "K_nu evals/s",
                          "workload": "100,000 pairs, x log-uniform [1e-3,140], nu U[0.05,10]",
                          "with_grad_value": grad_rate,
                          "with_grad_unit": "(K, dK/dx, dK/dnu) evals/s"},
            "probe": probe,
            "forms": forms,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
