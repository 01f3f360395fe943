"""Host logic of bench.py that needs no GPU: the CPU leg's comparison of GPU
output samples with the oracle, the FP32 forms' roofline from the committed
instruction counts, and the kernel-source hashes that key the ncu records."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2502_00356_gb300 import inputs  # noqa: E402


def test_oracle_checks_measure_the_planted_error():
    """Samples equal to the oracle give 0 error; a planted relative error of
    3e-6 on one entry (and 2e-12 absolute on a headline entry) is what the
    check reports."""
    x, nu = inputs.kv_pairs(40, seed=3, nu_lo=0.05, nu_hi=20.0)
    kx = oracle.besselk_f64(x, nu)
    locs = inputs.morton_sorted(inputs.jittered_grid(60, seed=4))
    I, J = inputs.entry_sample(60, 50, seed=5, near_fraction=0.1)
    m32 = oracle.matern_entries_f64(locs, I, J, 1.2, 0.08, 1.7)
    bad = m32.copy()
    bad[7] *= 1.0 + 3e-6
    mh = oracle.matern_entries(locs, I, J, bench.SIGMA2, bench.BETA, 0.5)
    mh_bad = mh.copy()
    mh_bad[3] += 2e-12
    samples = [{"key": "learned_eval", "kind": "eval", "x": x, "nu": nu, "got": kx},
               {"key": "fp32_matern", "kind": "matern", "locs": locs, "I": I, "J": J,
                "theta": (1.2, 0.08, 1.7), "got": bad}]
    out, secs = bench.oracle_checks(samples, {0.5: (locs, I, J, mh_bad)})
    assert out["learned_eval"]["max_rel_vs_oracle"] == 0.0
    assert out["learned_eval"]["sample"] == 40
    assert abs(out["fp32_matern"]["max_rel_vs_oracle"] - 3e-6) < 1e-9
    assert abs(out["plain_fp64"]["max_abs_vs_oracle"] - 2e-12) < 1e-15
    assert out["plain_fp64"]["sample"] == 50 and secs >= 0.0


def test_issue_roofline_from_the_committed_counts(monkeypatch):
    rec = {"kernel_hash": bench.kernel_hash(bench.FP32_SOURCES),
           "kernels": {"learned_matern": {"thread_inst": 4.0e11, "warp_inst": 1.3e10}}}
    monkeypatch.setattr(bench, "profiled_instr", lambda: rec)
    r = bench.issue_roofline("learned_matern", "k", 0.02, 8.0e8)
    assert r["achieved"] == pytest.approx(4.0e11 / 0.02 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.ISSUE_PEAK_GINST)
    assert r["thread_inst_per_eval"] == pytest.approx(500.0)
    assert r["lanes_active_of_32"] == pytest.approx(4.0e11 / 1.3e10)
    assert bench.issue_roofline("fp32_eval_L4", "k", 0.01, 1e8)["achieved"] is None


def test_recorded_profiles_match_their_sources_or_are_ignored():
    """A committed ncu record is used only while its kernel-source hash
    matches; the hashes ignore comments."""
    for name, files in (("matern_sym_f64_traffic.json", bench.KERNEL_SOURCES),
                        ("fp32_forms_instr.json", bench.FP32_SOURCES)):
        with open(os.path.join(ROOT, "profiles", name)) as f:
            rec = json.load(f)
        assert len(rec["kernel_hash"]) == 16
    assert bench.kernel_hash() == bench.kernel_hash(bench.KERNEL_SOURCES)
    assert bench.kernel_hash(bench.FP32_SOURCES) != bench.kernel_hash()
    assert bench.ISSUE_PEAK_GINST == pytest.approx(152 * 4 * 32 * 2.07)
    assert bench.FP64_PEAK_GOPS == pytest.approx(152 * 2 * 2.07)
