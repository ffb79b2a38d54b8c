"""The measured arithmetic peaks used as roofline denominators.

tsm_measure_fma_peak times a register-resident FMA loop; on a GB300 the FP32
rate must lie between half and 1.1x the nominal 80.5 TFLOP/s (152 SMs x 128
lanes x 2 flop x 2.07 GHz) and the FP64 rate far below it (GB300's FP64 pipe
is narrow), and the call leaves the current device unchanged."""
import pytest

from paper_1211_0126_gb300 import tsm

pytestmark = pytest.mark.gpu


def test_fma_peaks(libtsm):
    import torch
    dev = torch.cuda.current_device()
    f32 = tsm.tsm_measure_fma_peak(dev, tsm.TSM_F32)
    f64 = tsm.tsm_measure_fma_peak(dev, tsm.TSM_F64)
    print("FMA peaks: FP32 %.1f TFLOP/s, FP64 %.2f TFLOP/s" % (f32, f64))
    assert 0.5 * 80.5 < f32 < 1.1 * 80.5
    assert 0.0 < f64 < 0.25 * f32
    assert torch.cuda.current_device() == dev
    with pytest.raises(tsm.TsmError):
        tsm.tsm_measure_fma_peak(dev, tsm.TSM_F16)
