"""The throughput probes behind the roofline denominators (laps_measure_peaks):
the values are those of a GPU of this class at its running clock, not noise."""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2601_16696_gb300 import build, laps
    build.build()
    laps.lib()
    return laps


def test_measure_peaks_plausible(L):
    p = L.measure_peaks()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    assert p["sm_count"] == nsm
    assert 500.0 < p["sm_mhz"] < 3500.0
    # FFMA: 128 lanes x 2 FLOP per clock per SM, at most; a probe well below half
    # of that would not measure the pipe
    fp32_max = nsm * 256 * p["sm_mhz"] * 1e6 / 1e12
    assert 0.5 * fp32_max < p["fp32_tflops"] <= 1.05 * fp32_max, (p, fp32_max)
    assert 0.0 < p["fp64_tflops"] < p["fp32_tflops"]
    assert 1.0 <= p["ex2_per_clk_sm"] <= 64.0
    assert 0.05 < p["grid_barrier_us"] < 100.0 and p["barrier_blocks"] == nsm
