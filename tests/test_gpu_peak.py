"""The measured-peak entry point (bem_measure_peak), the denominator of the ALU rooflines: it
reports the device's multiprocessor count, positive rates for the FFMA, FFMA2 and DFMA chains
that grow with the work (the chains are not optimised away: twice the iterations take about
twice the time), and it refuses unknown kinds and sizes."""
import pytest

pytestmark = pytest.mark.gpu


def test_measured_peaks():
    import torch
    import paper_1511_04355_gb300 as P
    c = P.Context(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    r32, ms32, n = P.bem_measure_peak(c.h, P.BEM_PEAK_FP32, 256, 3)
    r32b, ms32b, _ = P.bem_measure_peak(c.h, P.BEM_PEAK_FP32, 512, 3)
    r2, _, _ = P.bem_measure_peak(c.h, P.BEM_PEAK_FP32X2, 256, 3)
    r64, _, _ = P.bem_measure_peak(c.h, P.BEM_PEAK_FP64, 64, 3)
    print(f"FP32 {r32:.1f} / {r32b:.1f}, FP32x2 {r2:.1f}, FP64 {r64:.2f} TFLOP/s on {n} SMs")
    assert n == sms
    assert r32 > 0 and r2 > 0 and r64 > 0
    assert 1.6 < ms32b / ms32 < 2.4
    assert r32 > 10 * r64
    for kind, it, reps in ((7, 16, 1), (P.BEM_PEAK_FP32, 0, 1), (P.BEM_PEAK_FP32, 16, 0)):
        with pytest.raises(P.BemError) as e:
            P.bem_measure_peak(c.h, kind, it, reps)
        assert e.value.code == P.BEM_ERR_INVALID_ARG
