"""Host-side bookkeeping of the benchmark line (no GPU): timing classes summed
per kernel function, the dominant kernel's roofline entry against the peak of
its precision form, the DRAM traffic scaled to a mean launch, and the
converged-point count."""
import importlib.util
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    # fixed peaks, whatever the machine's measurement file holds
    mod.measured_peaks = lambda: ({"hbm_gbs": 7000.0, "bf16_tflops": 1900.0,
                                   "bf16_tflops_sustained": 1800.0}, "test")
    return mod


def _timing():
    # ms, launches, algorithmic FP64-equivalent flops per class
    return {
        "tc_gemm_K": {"ms": 100.0, "launches": 10, "flops": 3.0e13, "bytes": 0.0},
        "tc_gemm_T1_dscale": {"ms": 300.0, "launches": 10, "flops": 1.2e14, "bytes": 0.0},
        "tc_gemm_T2": {"ms": 300.0, "launches": 10, "flops": 1.2e14, "bytes": 0.0},
        "tc_alpha_beta": {"ms": 50.0, "launches": 10, "flops": 0.5e13, "bytes": 0.0},
        "tc_alpha_dot": {"ms": 50.0, "launches": 10, "flops": 0.5e13, "bytes": 0.0},
        "emu_gemm_T1": {"ms": 200.0, "launches": 2, "flops": 1.0e13, "bytes": 0.0},
        "emu_gemm_T2": {"ms": 200.0, "launches": 2, "flops": 1.0e13, "bytes": 0.0},
        "gmres_step": {"ms": 40.0, "launches": 20, "flops": 0.0, "bytes": 0.0},
        "gmres_select": {"ms": 1.0, "launches": 0, "flops": 0.0, "bytes": 0.0},
    }


def test_classes_are_summed_per_kernel_function(bench):
    k = bench.per_kernel(_timing())
    assert k["gemm_tc_kernel"]["ms"] == pytest.approx(800.0)
    assert k["gemm_tc_kernel"]["launches"] == 50
    assert k["gemm_tc_kernel"]["flops"] == pytest.approx(2.8e14)
    assert sorted(k["gemm_tc_kernel"]["classes"]) == sorted(
        ["tc_gemm_K", "tc_gemm_T1_dscale", "tc_gemm_T2", "tc_alpha_beta", "tc_alpha_dot"])
    assert k["ozaki_gemm_kernel"]["ms"] == pytest.approx(400.0)
    assert "gmres_select" not in k                # classes without launches are dropped


def test_roofline_entry_of_the_dominant_kernel(bench):
    r = bench.roofline_of(_timing(), step_ms=1241.0, prec="bf16x3emu")
    assert r["kernel"] == "gemm_tc_kernel"
    # 2.8e14 flops in 800 ms: 350 TFLOP/s against 1800 / 3 (three bf16 products)
    assert r["achieved"] == pytest.approx(350.0)
    assert r["peak"] == pytest.approx(600.0)
    assert r["frac"] == pytest.approx(350.0 / 600.0)
    assert r["share_of_step"] == pytest.approx(800.0 / 1241.0)
    # traffic: bytes per flop of the capture times the mean launch's flops
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_FLOP["gemm_tc_kernel"] * 2.8e14 / 50)


def test_peaks_follow_the_precision_form(bench):
    assert bench.kernel_peak("gemm_tc_kernel", "tf32emu")[1] == pytest.approx(1800.0 * 0.5)
    assert bench.kernel_peak("ozaki_gemm_kernel", "bf16x3emu")[1] == pytest.approx(1800.0 / 15)
    assert bench.kernel_peak("ozaki_gemm_kernel", "fp64emu")[1] == pytest.approx(1800.0 / 21)
    # the TF32 form has no traffic capture of its own
    r = bench.roofline_of(_timing(), step_ms=1241.0, prec="tf32emu")
    assert r["traffic"] is None


def test_kernel_table_rates(bench):
    t = bench.kernel_table(_timing(), "bf16x3emu")
    assert t["ozaki_gemm_kernel"]["tflops"] == pytest.approx(50.0)   # 2e13 flops in 0.4 s
    assert t["ozaki_gemm_kernel"]["frac"] == pytest.approx(50.0 / 120.0, abs=1e-4)
    assert "tflops" not in t["gmres_step_kernel"]


def test_converged_points_need_all_three_directions(bench):
    info = {"converged": np.array([[1, 1, 1], [1, 0, 1], [0, 0, 0], [1, 1, 1]], dtype=bool)}
    assert bench.converged_points(info) == (2, 2)
