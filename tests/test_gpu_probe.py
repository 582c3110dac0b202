"""The benchmark's FP32 FMA rate probe (libarprobe.so, not part of libar): a
plausible rate for one GB300 (nominal 152 SMs x 128 lanes x 2 flops x 2.07
GHz = 80.5 TFLOP/s), scalar and packed, and argument checks."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_fma_rate():
    from paper_2503_00308_gb300 import _build, probe
    _build.build()
    assert torch.cuda.is_available()
    for packed in (False, True):
        r = probe.fp32_fma_rate(packed, 4096)
        assert 20.0 < r < 120.0, r
    with pytest.raises(RuntimeError):
        probe.fp32_fma_rate(False, 0)
