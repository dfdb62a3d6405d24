"""The library's FMA-throughput kernel (dmn_peak_gflops), the denominator of the bench's
compute rooflines: its measured FP64 and FP32 rates lie near the rates the chip's unit
counts give (152 SMs x 4 x 0.5 DFMA and 152 x 128 FFMA per clock at 2.07 GHz), and below
them apart from clock and rounding slack."""
import pytest

from paper_2103_08253_gb300 import dmn

pytestmark = pytest.mark.gpu


def test_measured_fma_peaks_are_near_the_unit_count_rates():
    d64 = 152 * 4 * 0.5 * 2 * 2.07
    d32 = 152 * 128 * 2 * 2.07
    g64, ms64 = dmn.peak_gflops("fp64", 0.2)
    g32, ms32 = dmn.peak_gflops("fp32", 0.1)
    assert ms64 >= 150.0 and ms32 >= 70.0
    assert 0.7 * d64 <= g64 <= 1.02 * d64, g64
    assert 0.6 * d32 <= g32 <= 1.02 * d32, g32


def test_fp64_pipe_spends_a_warp_instruction_on_masked_lanes_and_needs_one_warp_per_partition():
    """The two facts the Newton kernels' mapping rests on: (1) the FP64 pipe takes as long for a
    warp instruction with 16 active lanes as with 32 (the rate of the active lanes halves), so a
    mapping that leaves lanes idle at the tree's upper levels pays for them in full; (2) one warp
    per SM sub-partition (4 per SM) with one dependent chain per thread already comes close to
    the peak, so a few resident warps hide the FP64 latency."""
    full, _ = dmn.fma_throughput("fp64", 16, 4, 32, 0.1)
    half, _ = dmn.fma_throughput("fp64", 16, 4, 16, 0.1)
    assert 0.45 <= half / full <= 0.55, (half, full)
    one_warp, _ = dmn.fma_throughput("fp64", 4, 1, 32, 0.1)
    peak, _ = dmn.peak_gflops("fp64", 0.2)
    assert one_warp >= 0.85 * peak, (one_warp, peak)
