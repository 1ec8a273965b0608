"""The arithmetic-peak probes behind the benchmark's roofline denominators: plausible,
self-consistent rates measured on the device (no compute of the method involved)."""
import pytest
import torch

from paper_2203_15963_gb300 import native

pytestmark = pytest.mark.gpu


def test_measured_peaks_are_consistent():
    native.build()
    native.load()
    p = native.blacklight_measure_peaks(reps=3)
    props = torch.cuda.get_device_properties(0)
    assert p["sm_count"] == props.multi_processor_count
    assert p["sm_clock_khz"] > 0
    # every probe ran and took measurable time
    assert p["fp64_tflops"] > 0 and p["fp32_tflops"] > 0 and p["df64_tflops"] > 0
    assert p["probe_ms"] > 0
    # an FP32 FMA is never slower than an FP64 one, and the double-float multiply-add (about
    # a dozen FP32 instructions) sits between native FP32 and a small fraction of it
    assert p["fp32_tflops"] >= p["fp64_tflops"]
    assert p["df64_tflops"] < p["fp32_tflops"] / 4
    # no probe exceeds what the SMs could issue at the maximum clock: 2 flops per FP32 lane
    # (128 lanes an SM) per cycle
    bound = p["sm_count"] * 128 * 2 * p["sm_clock_khz"] * 1e3 / 1e12
    assert p["fp32_tflops"] <= 1.05 * bound


def test_measure_peaks_rejects_bad_arguments():
    native.load()
    with pytest.raises(native.BlacklightError):
        native.blacklight_measure_peaks(reps=0)
