"""The pipe-peak microbenchmarks behind gd_measure_peaks.

The FP32 FMA rate can reach, and not pass, the SM count x 128 lanes x the part's top
SM clock: a rate above that would mean the compiler dropped the timed work, one far
below it a broken launch.  The shared-memory byte-load rate has no firm ceiling here
(one warp-wide load per SM per clock is the nominal the roofline uses), so it gets
sanity bounds around that nominal.
"""
import pytest
import torch

from paper_1901_06229_b300 import geodock as gdk

pytestmark = pytest.mark.gpu


def top_sm_mhz() -> float:
    try:
        import pynvml
        pynvml.nvmlInit()
        try:
            h = pynvml.nvmlDeviceGetHandleByIndex(torch.cuda.current_device())
            return float(pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM))
        finally:
            pynvml.nvmlShutdown()
    except Exception:
        return 2032.0  # B300's top SM clock


def test_measured_pipe_peaks_are_physical():
    p = gdk.measure_peaks(torch.cuda.current_device())
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = top_sm_mhz()
    ffma_top = sms * 128 * mhz * 1e6
    lds_nominal = sms * 32 * mhz * 1e6
    assert 0.5 * ffma_top < p["ffma_per_s"] <= 1.02 * ffma_top, (p, mhz)
    assert 0.25 * lds_nominal < p["lds_u8_per_s"] < 4.0 * lds_nominal, (p, mhz)


def test_measure_peaks_on_a_side_stream_leaves_no_error_behind():
    s = torch.cuda.Stream()
    p = gdk.measure_peaks(torch.cuda.current_device(), stream=s)
    assert p["ffma_per_s"] > 0 and p["lds_u8_per_s"] > 0
    x = torch.ones(1024, device="cuda")
    assert float(x.sum()) == 1024.0  # the context is healthy afterwards
