"""The roofline arithmetic of bench.py, on CPU.

  * The split-radix operation count S(L) = 4 L log2 L - 6 L + 8 reproduces
    the published minimal real-operation counts of the split-radix FFT for 8
    and 16 points (56 and 168: 4 + 52 and 24 + 144 multiplies + adds).
  * The per-kernel transform flops and algorithmic bytes at n = 256 are the
    figures the roofline line reports (26.40 GFLOP for the y/z executor,
    30.8 GFLOP per solve, 3.42 GFLOP per field-direction; 0.606 / 1.281 /
    1.211 GB per kernel; B_io 671.9 MB, B_method 3097 MB).
  * The derived FP32 peak is 152 SMs x 128 lanes x 2 flops x 2070 MHz.
"""
import math

import pytest

import bench


def split_radix(L):
    return 4 * L * math.log2(L) - 6 * L + 8


@pytest.mark.parametrize("L,ops", [(8, 56), (16, 168)])
def test_split_radix_count_matches_the_published_minimum(L, ops):
    assert split_radix(L) == ops


def test_transform_flops_at_256():
    fl = bench.transform_flops(256)
    assert fl["yz_executor"] == pytest.approx(26.404e9, rel=1e-4)
    total = sum(fl.values())
    assert total == pytest.approx(30.79e9, rel=1e-3)
    # nine field-directions per solve (3 forward, 6 inverse)
    assert total / 9 == pytest.approx(3.42e9, rel=2e-3)
    # the x parts are real lines: half a complex pruned line each
    assert fl["x_inverse"] == pytest.approx(2 * fl["x_forward"])


def test_kernel_and_method_bytes_at_256():
    kb = bench.kernel_bytes(256)
    assert kb["x_forward"] == 605_552_640
    assert kb["yz_executor"] == 1_280_576_516
    assert kb["x_inverse"] == 1_211_105_280
    b_io, b_method = bench.algorithmic_bytes(256)
    assert b_io == 671_878_148
    assert b_method == 3_097_234_436


def test_derived_fp32_peak():
    # 152 SMs (the count bench.py reads from the device) x 128 lanes x 2 flop x 2070 MHz
    peak = 152 * bench.FP32_LANES_PER_SM * 2 * 2070e6
    assert peak == pytest.approx(80.548e12, rel=1e-4)
