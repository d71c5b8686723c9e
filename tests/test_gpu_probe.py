"""Throughput probes: rates are positive and below what the device's unit counts allow."""
import pytest

from tests.gpu_common import cuda

pytestmark = pytest.mark.gpu


def test_probe_rates_within_unit_limits():
    torch, V = cuda()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    ghz = 2.2                                   # above any SM clock of the part
    ffma = V.probe_rate(V.PROBE_FFMA, 7)
    assert 0 < ffma <= sms * 128 * ghz * 1e9
    for pr in (V.PROBE_RSQRT, V.PROBE_EX2):
        r = V.probe_rate(pr, 7)
        assert 0 < r <= sms * 128 * ghz * 1e9
    pairs = V.probe_rate(V.PROBE_PAIRS_T4, 7)
    assert 0 < pairs <= ffma / 8 * 1.05         # at least 8 FP32 operations per pair
    # one evaluation (11 FP32 operations) serves two pairs across rows
    sym = V.probe_rate(V.PROBE_PAIRS_SYM, 7)
    assert 0 < sym <= ffma / 5.5 * 1.05
    with pytest.raises(V.VpmError):
        V.probe_rate(V.PROBE_PAIRS_T4, 9)
