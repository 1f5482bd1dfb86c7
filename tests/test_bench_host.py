"""Host-side arithmetic of bench.py (no GPU): the roofline entries and the
derived peak of the mixed-path recompute."""
import dataclasses
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_mixed_recompute_peak_is_the_fp32_issue_bound():
    import bench
    instr = 152 * 128 * 2.07e9
    residual = instr * 2 / 11 / 1e12      # double-float multiply-add: 2 flop in 11 instructions
    correction = instr * 2 / 1e12         # FP32 FMA: 2 flop per instruction
    assert bench.MIXED_RECOMPUTE_TFLOPS == pytest.approx(4.0 / (2.0 / residual + 2.0 / correction))
    assert 13.0 < bench.MIXED_RECOMPUTE_TFLOPS < 14.0


def test_roofline_entries():
    import bench
    from paper_1901_01047_gb300 import inputs
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
    mixed = inputs.WORKLOADS["batched256"]
    fp64 = inputs.WORKLOADS["betts16"]
    work = {"update": (6.8e9, 13.6e9), "recompute": (None, 2.0e12)}
    r = bench.roofline("update", 2000.0, 10, work, peaks, "measured", mixed)  # 2 s for 6.8 GB
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(3.4) and r["frac"] == pytest.approx(3.4 / 6800.0)
    assert r["launch_ms"] == pytest.approx(200.0)
    assert r["tf32_peak_tflops"] == pytest.approx(1900.0 * 1.1 / 2.25)
    # mixed path, residual from digit planes: 17 FP16 products at the 16-bit
    # tensor rate plus the FP32 correction, 4n^3 flop in all
    r = bench.roofline("recompute", 1000.0, 10, work, peaks, "measured", mixed)
    assert r["bound"] == "tensor" and r["achieved"] == pytest.approx(2.0)
    fp32 = 152 * 128 * 2.07e9 * 2 / 1e12
    assert r["peak"] == pytest.approx(4.0 / (2.0 * 17 / 1900.0 + 2.0 / fp32))
    peaks_s = dict(peaks, bf16_tflops_sustained=1700.0)
    r = bench.roofline("recompute", 1000.0, 10, work, peaks_s, "measured", mixed)
    assert r["peak"] == pytest.approx(4.0 / (2.0 * 17 / 1700.0 + 2.0 / fp32))
    # the double-float residual: FP32 issue bound
    r = bench.roofline("recompute", 1000.0, 10, work, peaks, "measured", dataclasses.replace(mixed, recompute_method="newton_df"))
    assert r["bound"] == "alu" and r["peak"] == pytest.approx(bench.MIXED_RECOMPUTE_TFLOPS)
    r = bench.roofline("recompute", 1000.0, 10, work, peaks, "measured", fp64)
    assert r["peak"] == pytest.approx(bench.FP64_TFLOPS)
    r = bench.roofline("metropolis", 1000.0, 10, work, peaks, "measured", mixed)
    assert r["bound"] is None and r["frac"] is None


def test_workload_overrides():
    import argparse
    import bench
    args = argparse.Namespace(workload="batched256", schedule="lockstep", duplicate_rule="abort", walkers=32)
    wl = bench.workload_of(args)
    assert wl.walkers == 32 and wl.schedule == "lockstep" and wl.duplicate_rule == "abort"
    params, wp = wl.problem_params()
    full, _ = bench.workload_of(argparse.Namespace(workload="batched256")).problem_params()
    assert len(params) == 32 and params == full[:32]  # the first walkers' problems of the full batch
