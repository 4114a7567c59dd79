"""The FFMA-rate probe (bf_measure_ffma), the peak that the plain FP32
form's roofline fraction divides by: its rate must be that of 128 FP32 lanes
per SM at a clock the GPU can run, and bad arguments must be refused."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1412_4907_gb300 as m
    return m


def test_ffma_probe_rate(bf):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2 * 2.2e9 / 1e12   # every lane, one FFMA per cycle, at 2.2 GHz
    tf = bf.bf_measure_ffma(0.2)
    assert 0.3 * ceiling < tf < ceiling, (tf, ceiling)


@pytest.mark.parametrize("seconds", [0.0, -1.0, 61.0])
def test_ffma_probe_rejects_bad_durations(bf, seconds):
    with pytest.raises(bf.BFError) as ei:
        bf.bf_measure_ffma(seconds)
    assert ei.value.status == bf.BF_ERR_ARG
