"""The library's roofline probes: the measured binary32 and binary64 FMA
rates and the L2 read bandwidth are positive, bounded by what the device's
SM count and clock allow, and in the order the hardware fixes."""
import pytest

pytestmark = pytest.mark.gpu

from paper_1307_2643_gb300 import crp  # noqa: E402


def test_measured_peaks_are_plausible():
    import torch
    from paper_1307_2643_gb300.build import build
    build()
    pk = crp.crp_measure_peaks(0)
    props = torch.cuda.get_device_properties(0)
    assert pk["sm_count"] == props.multi_processor_count
    assert pk["l2_bytes"] > 0
    # at most 128 binary32 FMA lanes per SM at 2.2 GHz
    assert 0.2 * pk["sm_count"] * 128 * 2 * 1.0e9 / 1e12 < pk["fp32_tflops"]
    assert pk["fp32_tflops"] < pk["sm_count"] * 128 * 2 * 2.2e9 / 1e12
    assert 0.0 < pk["fp64_tflops"] < pk["fp32_tflops"]
    assert pk["l2_read_gbs"] > 1000.0
    with pytest.raises(crp.CrpError):
        crp.crp_measure_peaks(-1)
