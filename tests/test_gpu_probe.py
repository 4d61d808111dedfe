"""The throughput probes behind the integer roofline (GPU): every mode
returns a positive rate per SM cycle and the SM count; the raw DPX rate
bounds the shipped cell sequence, which issues at least four DPX operations
per cell pair."""
import pytest

pytestmark = pytest.mark.gpu


def test_probe_modes(gpu):
    dpx, sms = gpu.sw_probe_alu_rate(0, 0)
    cells16, sms1 = gpu.sw_probe_alu_rate(0, 1)
    cells8, sms2 = gpu.sw_probe_alu_rate(0, 2)
    assert sms == sms1 == sms2 > 0
    assert dpx > 0 and cells16 > 0 and cells8 > 0
    assert cells16 <= dpx / 2.0 * 1.05
    cells2, _ = gpu.sw_probe_alu_rate(0, 3)
    assert 0 < cells2 <= dpx / 2.0 * 1.05
    with pytest.raises(gpu.SwError):
        gpu.sw_probe_alu_rate(0, 4)
