"""Host-side arithmetic of bench.py's JSON line (no GPU): the whole-job value,
the sweep's HBM floor and the roofline rows it reports per kernel class."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PEAKS = {"hbm_gbs": 6779.0, "bf16_tflops": 1918.8}


def test_job_value_counts_every_rank(bench):
    # 400 sweeps on each of 2 replicas in 1 s of the slowest rank
    assert bench.job_value(400, 2, 1000.0) == pytest.approx(800.0)
    assert bench.job_value(20, 1, 10.0) == pytest.approx(2000.0)


def test_sweep_floor_bytes_256x256x31x8(bench):
    dims = (256, 256, 31, 8)
    P = 256 * 256 * 31 * 8
    # N + 2 FP32 passes over X and one mask bit per element
    assert bench.sweep_floor_bytes(dims, None) == pytest.approx(6 * 4 * P + P / 8)
    assert bench.sweep_floor_bytes(dims, None) == pytest.approx(392101888.0)


def test_hbm_class_rate_is_bytes_per_launch_over_launch_time(bench):
    prof = {"launches": 4, "ms": 0.4, "bytes": 4.0e8, "flops": 0.0}
    row = bench.class_roofline("xupdate", prof, PEAKS, "measured", "fp32", [216] * 4, 0)
    assert row["bound"] == "hbm" and row["unit"] == "GB/s"
    # 1e8 bytes per launch in 0.1 ms
    assert row["achieved"] == pytest.approx(1000.0)
    assert row["frac"] == pytest.approx(1000.0 / 6779.0)
    assert row["bytes_per_launch"] == pytest.approx(1.0e8)


def test_tensor_rate_uses_the_tf32_half_of_the_bf16_peak(bench):
    prof = {"launches": 2, "ms": 0.2, "bytes": 2.0e8, "flops": 2.0e10}
    row = bench.class_roofline("gram", prof, PEAKS, "measured", "tf32", [216] * 4, 0)
    # 1e10 flops per launch in 0.1 ms = 100 TFLOP/s against 959.4
    assert row["tensor_tflops"] == pytest.approx(100.0)
    assert row["tensor_frac"] == pytest.approx(100.0 / (0.5 * 1918.8))


def test_contraction_classes_follow_the_precision(bench):
    prof = {"launches": 5, "ms": 0.1, "bytes": 5.0e8, "flops": 1.0e9}
    tc = bench.class_roofline("rhs2", prof, PEAKS, "measured", "tf32", [216] * 4, 0)
    assert tc["kernel"].startswith("k_tcc") and tc["bound"] == "hbm"
    fp = bench.class_roofline("rhs2", prof, PEAKS, "measured", "fp32", [216] * 4, 0)
    assert fp["kernel"].startswith("k_sgemm") and fp["bound"] == "alu" and fp["unit"] == "TFLOP/s"
    # 2e8 flops per launch in 20 us
    assert fp["achieved"] == pytest.approx(10.0)


def test_factorization_rate_per_occupied_sm(bench):
    dims = (256, 256, 31, 8)
    prof = {"launches": 4, "ms": 0.2, "bytes": 0.0, "flops": 0.0}
    row = bench.class_roofline("eig", prof, PEAKS, "measured", "tf32", [216] * 4, 0, dims=dims)
    groups = [I // 2 + 1 for I in dims]  # one CTA per distinct shift
    flops = np.mean([g * 216 ** 3 / 3.0 for g in groups])
    sms = np.mean([min(g, 152) for g in groups])
    assert row["flops_per_launch"] == pytest.approx(flops)
    assert row["achieved"] == pytest.approx(flops / 50e-6 / 1e12)
    assert row["peak"] == pytest.approx(sms * bench.SM_FP32_TFLOPS)
    assert row["frac"] == pytest.approx(row["achieved"] / row["peak"])
