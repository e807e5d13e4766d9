"""The arithmetic-pipe microbenchmarks (lr_measure_peak) return rates in the
range the unit counts allow: at most 152 SMs x (128 FP32 FMA | 2 FP64 FMA) per
clock x 2 flops x the 2.07 GHz maximum SM clock, and for TF32 152 SMs x 4096
dense TF32 flops per clock (half the bf16 rate, 2.25 PFLOP/s nominal) x 2.07 GHz,
each plus 5% for timing slack; at least 40% of it (a busy or power-capped GPU
still reaches that)."""
import pytest

from paper_2508_18114_gb300 import lr

pytestmark = pytest.mark.gpu

CEIL = {"fp32_fma": 152 * 128 * 2 * 2.07e9, "fp64_fma": 152 * 2 * 2 * 2.07e9, "tf32_mma": 152 * 4096 * 2.07e9}


@pytest.mark.parametrize("kind", ["fp32_fma", "fp64_fma", "tf32_mma"])
def test_measured_peak_in_range(kind):
    f, sec = lr.measure_peak(kind)
    print(kind, "%.3e flop/s in %.3f ms" % (f, sec * 1e3))
    assert sec > 0
    assert 0.4 * CEIL[kind] < f < 1.05 * CEIL[kind]
