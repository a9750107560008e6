"""The shared-memory bandwidth probe (the denominator of the shared-memory
step kernel's roofline): a plausible figure for the device, and argument
errors reported without a launch."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mq():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2605_06921_gb300 as m
    return m


def test_smem_probe_is_plausible(mq):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    gbs = mq.measure_smem_gbs()
    # 128 bytes per clock per SM at 1.0 to 2.2 GHz, with room on both sides
    lo, hi = 0.5 * 128 * sms * 1.0, 1.2 * 128 * sms * 2.2
    assert lo < gbs < hi, gbs
    # longer runs agree within the noise of the clock
    assert abs(mq.measure_smem_gbs(8192) / gbs - 1.0) < 0.2


def test_smem_probe_rejects_bad_arguments(mq):
    with pytest.raises(mq.MqoError):
        mq.measure_smem_gbs(0)
