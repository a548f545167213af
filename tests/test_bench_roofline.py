"""The roofline arithmetic behind bench.py's `roofline` and `kernels` objects,
on the CPU: the method's work per launch against closed forms, and the
fraction of a launch that takes exactly its roof time."""
import math
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_forward_work_is_one_exp_per_pair_and_the_two_contractions():
    n, d, m = 65536, 8, 16
    e, fl, ops = bench.kernel_work("bf16_hilo", "fwd", d, m, n)
    assert e == n * n
    assert fl == n * n * (2 * d + 2 * m)
    assert ops == 0
    # the one-column CG product counts the same way with m = 1
    e1, fl1, _ = bench.kernel_work("bf16_hilo", "fwd_m1", d, 1, n)
    assert (e1, fl1) == (n * n, n * n * (2 * d + 2))


def test_adjoint_work_counts_the_symmetric_half_once():
    n, d, m = 1000, 3, 2
    e, fl, _ = bench.kernel_work("bf16_hilo", "adj", d, m, n)
    half = n * (n + 1) // 2
    assert e == half == sum(range(1, n + 1))
    assert fl == half * (2 * d + 4 * m + 2 * (2 * d + 1))


def test_fp32_forms_are_counted_on_the_fma_pipe():
    n, d, m = 512, 4, 3
    assert bench.kernel_work("fp32", "fwd", d, m, n) == (0, 0, n * n * (2 * d + m))
    assert bench.kernel_work("fp32", "adj", d, m, n) == (0, 0, n * n * (4 * d + 2 * m + 2))


def test_a_launch_at_its_roof_time_has_fraction_one():
    n, d, m, mhz = 65536, 8, 16, 2070.0
    roof_ms = n * n / (bench.SM_COUNT * bench.MUFU_EX2_LANES * mhz * 1e6) * 1e3
    r = bench.kernel_roof("bf16_hilo", "fwd", d, m, n, mhz, 2000.0, roof_ms)
    assert r["bound"] == "alu" and r["unit"] == "G ex2/s"
    assert r["peak"] == pytest.approx(152 * 32 * 2.07, rel=1e-12)
    assert r["frac"] == pytest.approx(1.0, rel=1e-12)
    assert r["roof_ms"] == pytest.approx(roof_ms, rel=1e-12)
    # twice the time, half the fraction
    assert bench.kernel_roof("bf16_hilo", "fwd", d, m, n, mhz, 2000.0, 2 * roof_ms)["frac"] == pytest.approx(0.5)


def test_the_binding_unit_is_the_slowest_one():
    n, d, m, mhz = 4096, 8, 64, 2070.0
    # a tensor peak so low that the contractions take longer than the exps
    r = bench.kernel_roof("bf16_hilo", "fwd", d, m, n, mhz, 1e-3, 1.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    fl = n * n * (2 * d + 2 * m)
    assert r["roof_ms"] == pytest.approx(fl / 1e9 * 1e3, rel=1e-12)
    # the FP32 form: FMA-pipe operations
    r32 = bench.kernel_roof("fp32", "fwd", d, m, n, mhz, 2000.0, 1.0)
    assert r32["unit"] == "G FMA-pipe op/s"
    assert r32["peak"] == pytest.approx(bench.SM_COUNT * bench.FMA_LANES * mhz * 1e6 / 1e9)


def test_aggregate_rate_is_all_ranks_units_over_the_slowest_time():
    assert bench.aggregate_rate(2e9, 4, 1000.0) == pytest.approx(8.0)
    assert math.isclose(bench.aggregate_rate(1e9, 1, 500.0), 2.0)
