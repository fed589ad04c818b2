"""The measured FMA rates the rooflines are quoted against: each is close to
the unit count x clock of its precision, and paired FP32 FMA instructions do
the same FMA work per second as scalar ones (they halve the instructions,
not the pipe cycles)."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pa():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08374_gb300 as pa
    return pa


def test_fma_rates_near_the_derived_peaks(pa):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # flop/clk/SM: FP64 2 FMA x 2, FP32 128 FMA x 2; clocks between 1.0 and
    # 2.2 GHz cover any clock the part runs at under load
    f64 = pa.pa_measure_fma_rate(pa.PA_FP64)
    f32 = pa.pa_measure_fma_rate(pa.PA_FP32)
    f32x2 = pa.pa_measure_fma_rate(pa.PA_FMA_FP32X2)
    assert sms * 4 * 1.0e9 / 1e12 <= f64 <= sms * 4 * 2.2e9 / 1e12
    assert sms * 256 * 1.0e9 / 1e12 <= f32 <= sms * 256 * 2.2e9 / 1e12
    assert 0.8 * f32 <= f32x2 <= 1.25 * f32
