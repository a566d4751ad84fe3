"""The ceiling microbenchmarks the benchmark reports beside the roofline run
and give figures in the range GB300's units allow."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_ceilings_are_plausible():
    import bench
    c = bench.measure_ceilings(reps=2)
    assert "error" not in c, c
    assert c["sms"] > 0 and c["clock_mhz"] > 0
    # per clock per SM: FP64 FMAs at most one per lane of four sub-cores,
    # 32-bit IMADs at most 128 lanes, shared-memory loads at most 32 lanes
    # (one 128-byte wavefront per clock)
    assert 0.5 <= c["dfma_per_clk_sm"] <= 128
    assert 8 <= c["imad_per_clk_sm"] <= 130
    assert 1 <= c["lds_random_lanes_per_clk_sm"] <= c["lds_linear_lanes_per_clk_sm"] * 1.05
    assert c["lds_linear_lanes_per_clk_sm"] <= 33
