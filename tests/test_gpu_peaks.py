"""The issue-rate probe the bench's rooflines use (tde_measure_peaks)."""
import pytest
import torch

from paper_2509_19974_gb300 import tde

pytestmark = pytest.mark.gpu


def test_measure_peaks_is_plausible():
    """Rates per SM per clock: a tcgen05 M=128 N=256 MMA retires at most one
    per 64 cycles (E4M3: 128 x 256 x 32 MACs, E2M1: K = 64), the FP4 rate is
    the FP8 rate doubled or more, and POPC / IMAD do at most 128 results per
    clock (4 sub-partitions x 32 lanes)."""
    pk = tde.measure_peaks(0)
    assert pk["sm_count"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 2048 <= pk["e4m3_mac_per_sm_clk"] <= 16384 * 1.01
    assert pk["e2m1_mac_per_sm_clk"] >= 1.9 * pk["e4m3_mac_per_sm_clk"]
    assert 1 <= pk["popc_per_sm_clk"] <= 128 * 1.01
    assert 1 <= pk["imad_per_sm_clk"] <= 128 * 1.01
