"""Measured arithmetic ceilings (the roofline denominators of the pair loops):
each rate is positive and below what the SM count and the maximum clock
allow, and each pair term costs more than ten FP32 instructions."""
import pytest
import torch

from gpu_util import lib_ready

pytestmark = pytest.mark.gpu


def test_alu_ceilings_are_physical():
    voge = lib_ready()
    pk = voge.voge_measure_alu_peaks()
    torch.cuda.synchronize()
    sms = pk["sms"]
    assert sms == torch.cuda.get_device_properties(0).multi_processor_count
    clock_ghz = 2.2  # above the GB300's 2.07 GHz maximum SM clock
    fma_bound = sms * 128 * 2 * clock_ghz / 1e3  # TFLOP/s
    assert 0.3 * fma_bound < pk["fma_tflops"] < fma_bound
    assert 0.0 < pk["ex2_tops"] < sms * 32 * clock_ghz / 1e3  # at most 32 MUFU lanes per SM per clock
    # each pair is more than 10 FP32 instructions, so fewer than a tenth of the FMA lane rate
    lanes_per_s = sms * 128 * clock_ghz * 1e9
    for key in ("fwd_gpairs", "bwd_gpairs"):
        assert 0.0 < pk[key] * 1e9 < lanes_per_s / 10, (key, pk[key])
    assert all(t > 1.0 for t in pk["ms"])  # long enough to time with events
