"""The arithmetic behind bench.py's report, on the CPU: flops per pair (the projection P plus T
expansions plus the pair product, Hadamard product and accumulate), and the roofline object of
the dominant kernel (algorithmic flops over its live launch time, against the measured peak)."""
import math

import pytest

import bench


def test_flops_per_pair_is_t_plus_one_projections_plus_three_n_cubed():
    n, r, T = 96, 40, 40
    P = 2 * (n ** 3 * r + n ** 2 * r ** 2 + n * r ** 3)       # one projection: 112.6 MFLOP
    assert P == pytest.approx(112.6e6, rel=1e-3)
    assert bench.flops_per_pair(n, r, T) == (T + 1) * P + 3 * n ** 3
    assert bench.flops_per_pair(n, r, T) == pytest.approx(4.62e9, rel=1e-3)   # per distinct pair


def test_roofline_of_the_expansion_kernel():
    n, r, T, N, steps = 96, 40, 40, 64, 10
    launches, ms_total = 160, 162.17
    peaks = {"bf16_tflops_sustained": 1709.7}
    roof = bench.roofline("tc_consume", {"tc_consume": (launches, ms_total)}, n, r, T, N, steps, "bf16", peaks, None)
    unique = N * (N + 1) // 2
    flops = (T * 2 * (n ** 2 * r ** 2 + n ** 3 * r) + 3 * n ** 3) * unique * steps   # stages 2 and 3, epilogue
    assert roof["achieved"] == pytest.approx(flops / (ms_total / 1e3) / 1e12)
    assert roof["achieved"] == pytest.approx(514.8, rel=2e-3)                      # the reported bench value
    assert roof["peak"] == 1709.7 and roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == pytest.approx(roof["achieved"] / 1709.7)
    assert roof["avg_launch_ms"] == pytest.approx(ms_total / launches)
    # DRAM bytes per launch: the per-pair ncu figure times the pairs one launch processes
    per_pair = bench.DRAM_BYTES_PER_PAIR[("tc_consume", "bf16")]
    assert roof["traffic"] == pytest.approx(per_pair * unique * steps / launches)
    assert 20e6 < per_pair < 25e6


def test_roofline_peaks_per_precision():
    args = ("tc_consume", {"tc_consume": (10, 10.0)}, 32, 16, 30, 4, 1)
    peaks = {"bf16_tflops_sustained": 1700.0}
    assert bench.roofline(*args, "tf32", peaks, None)["peak"] == pytest.approx(850.0)
    assert bench.roofline(*args, "bf16", None, None)["peak_source"].startswith("fallback")
    assert bench.roofline(*args, "bf16", {"hbm_gbs": 6800.0}, None)["peak_source"].startswith("fallback")
    f = bench.roofline(*args, "fp32", peaks, None)
    assert f["bound"] == "alu"
    assert f["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)   # FP32 FMA rate of 152 SMs
    assert f["traffic"] is None                                          # no capture for this pair
    assert math.isfinite(f["frac"])
