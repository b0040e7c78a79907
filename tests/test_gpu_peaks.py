"""Measured ALU ceilings (felbm_alu_peak): plausible magnitudes for a GB300
(nominal FP64 1.25 TFLOP/s; FP32 152 SMs x 128 lanes x 2 flops x about
2 GHz, about 80 TFLOP/s) and the argument checks."""
import pytest

from paper_1608_01906_gb300 import felbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1608_01906_gb300 import build

    build.build()
    felbm.load()


def test_alu_peaks_plausible():
    fp32 = felbm.alu_peak(felbm.ALU_FP32)
    fp32x2 = felbm.alu_peak(felbm.ALU_FP32X2)
    fp64 = felbm.alu_peak(felbm.ALU_FP64)
    print("ALU peaks TFLOP/s: fp32 %.1f fp32x2 %.1f fp64 %.3f" % (fp32 / 1e12, fp32x2 / 1e12, fp64 / 1e12))
    assert 10e12 < fp32 < 300e12
    assert 10e12 < fp32x2 < 300e12
    assert 0.1e12 < fp64 < 10e12


def test_alu_peak_rejects_bad_kind():
    st, _ = felbm.felbm_alu_peak(3)
    assert st == felbm.FELBM_ERR_INVALID_ARG
