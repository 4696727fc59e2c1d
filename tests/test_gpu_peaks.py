"""The ALU throughput probe (hfmm_alu_peak) does the work it counts: its
measured rates lie within what the SM count and the clock allow.  Nominal
per-SM rates at the maximum SM clock: 128 FP32 lanes x 2 flop per cycle for
FMA; MUFU instructions at 16 per SM per cycle."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_probe_rates_are_physical():
    import torch

    from paper_2006_14952_gb300 import hfmm

    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    fmax_hz = 2.2e9  # above the GB300's 2070 MHz maximum SM clock
    fp32_bound = sms * 128 * 2 * fmax_hz
    ffma, t0 = hfmm.alu_peak("ffma", 1024)
    ffma2, t1 = hfmm.alu_peak("ffma2", 1024)
    ex2, _ = hfmm.alu_peak("ex2", 256)
    rsq, _ = hfmm.alu_peak("rsqrt", 256)
    print(f"ffma {ffma / 1e12:.1f} TFLOP/s ({t0:.2f} ms), ffma2 {ffma2 / 1e12:.1f} TFLOP/s ({t1:.2f} ms), "
          f"ex2 {ex2 / 1e12:.2f} Top/s, rsqrt {rsq / 1e12:.2f} Top/s")
    assert 0.25 * fp32_bound < ffma < 2.05 * fp32_bound
    assert 0.25 * fp32_bound < ffma2 < 2.05 * fp32_bound
    for r in (ex2, rsq):
        assert 0.01 * fp32_bound / 2 < r < fp32_bound / 2
