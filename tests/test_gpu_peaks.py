"""The issue-rate probe (dse_measure_peaks) against the part's documented
unit counts: 128 FP32 lanes, 16 (or 32) MUFU lanes and 2 FP64 FMA lanes per
SM per clock, at a clock between 0.5x and 1.05x the maximum SM clock the device
reports (the probe runs at whatever clock the part is at)."""
import pytest

import __graft_entry__ as ge

pytestmark = pytest.mark.gpu


def test_peaks_match_unit_counts():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ge.build()
    from paper_2602_06986_gb300 import dse

    p = dse.measure_peaks()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    mhz = getattr(props, "clock_rate", 0) / 1e3 or 2070.0
    # (MUFU lanes: 16 per SM for most functions; some parts issue ex2 at
    # twice that rate)
    for key, lanes, hi in (("fp32_fma_per_s", 128, 1.05), ("sfu_per_s", 16, 2.1), ("fp64_fma_per_s", 2, 1.05)):
        nominal = sms * lanes * mhz * 1e6
        assert 0.5 * nominal <= p[key] <= hi * nominal, (key, p[key], nominal)
    # the FP64 rate is a small fraction of the FP32 rate on this part
    assert p["fp64_fma_per_s"] < p["fp32_fma_per_s"] / 16
