"""The arithmetic behind bench.py's report, on the CPU: flops per pair (the projection P plus T
expansions plus the pair product, Hadamard product and accumulate), the pair counts of a target
block inside the occupied block, and the roofline object of the dominant kernel (algorithmic
flops over its live launch time, against the measured peak)."""
import math

import pytest

import bench


def test_flops_per_pair_is_t_plus_one_projections_plus_three_n_cubed():
    n, r, T = 96, 40, 40
    P = 2 * (n ** 3 * r + n ** 2 * r ** 2 + n * r ** 3)       # one projection: 112.6 MFLOP
    assert P == pytest.approx(112.6e6, rel=1e-3)
    assert bench.flops_per_pair(n, r, T) == (T + 1) * P + 3 * n ** 3
    assert bench.flops_per_pair(n, r, T) == pytest.approx(4.62e9, rel=1e-3)   # per distinct pair
    # the TiO2-shaped block: 37.6 GFLOP per distinct pair, ~16.5 PFLOP per apply
    assert bench.flops_per_pair(160, 64, 45) == pytest.approx(37.6e9, rel=2e-3)
    assert bench.flops_per_pair(160, 64, 45) * bench.pair_counts(1842, 256)[1] == pytest.approx(16.5e15, rel=5e-3)


def test_pair_counts_of_a_target_block_inside_the_occupied_block():
    assert bench.pair_counts(64, 64) == (4096, 2080)
    assert bench.pair_counts(1842, 256) == (471552, 471552 - 32640)
    assert bench.pair_counts(10, 3, subset=False) == (30, 30)


def test_roofline_of_the_expansion_kernel(monkeypatch):
    n, r, T, N, steps = 96, 40, 40, 64, 10
    unique = N * (N + 1) // 2
    launches, ms_total = 160, 162.17
    peaks = {"bf16_tflops_sustained": 1709.7}
    monkeypatch.setitem(bench.DRAM_BYTES_PER_PAIR, ("tc_consume", "bf16", "pt"), 22.0e6)
    roof = bench.roofline("tc_consume", {"tc_consume": (launches, ms_total)}, n, r, T, unique, steps, "bf16", peaks,
                          None, "pt")
    flops = (T * 2 * (n ** 2 * r ** 2 + n ** 3 * r) + 3 * n ** 3) * unique * steps   # stages 2 and 3, epilogue
    assert roof["achieved"] == pytest.approx(flops / (ms_total / 1e3) / 1e12)
    assert roof["achieved"] == pytest.approx(514.8, rel=2e-3)
    assert roof["peak"] == 1709.7 and roof["bound"] == "tensor" and roof["unit"] == "TFLOP/s"
    assert roof["frac"] == pytest.approx(roof["achieved"] / 1709.7)
    assert roof["avg_launch_ms"] == pytest.approx(ms_total / launches)
    # DRAM bytes per launch: the per-pair ncu figure times the pairs one launch processes
    assert roof["traffic"] == pytest.approx(22.0e6 * unique * steps / launches)
    # no capture for another workload: no traffic figure
    assert bench.roofline("tc_consume", {"tc_consume": (launches, ms_total)}, n, r, T, unique, steps, "bf16", peaks,
                          None, "batch")["traffic"] is None
    # the TiO2-shaped capture: 164 pairs in one launch, 22.16 GB read and 1.95 GB written
    assert bench.DRAM_BYTES_PER_PAIR[("tc_consume", "bf16", "tio2")] == pytest.approx(24.117e9 / 164, rel=1e-3)


def test_roofline_peaks_per_precision():
    args = ("tc_consume", {"tc_consume": (10, 10.0)}, 32, 16, 30, 10, 1)
    peaks = {"bf16_tflops_sustained": 1700.0}
    assert bench.roofline(*args, "tf32", peaks, None)["peak"] == pytest.approx(850.0)
    assert bench.roofline(*args, "bf16", None, None)["peak_source"].startswith("fallback")
    assert bench.roofline(*args, "bf16", {"hbm_gbs": 6800.0}, None)["peak_source"].startswith("fallback")
    f = bench.roofline(*args, "fp32", peaks, None)
    assert f["bound"] == "alu"
    assert f["peak"] == pytest.approx(152 * 128 * 2 * 2070e6 / 1e12)   # FP32 FMA rate of 152 SMs
    assert f["traffic"] is None                                          # no capture for this pair
    assert math.isfinite(f["frac"])
