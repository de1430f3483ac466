"""The measured arithmetic rates that the rooflines divide by (h2_measure_peak)."""
import pytest

torch = pytest.importorskip("torch")
h2 = pytest.importorskip("paper_2109_05451_gb300")

pytestmark = pytest.mark.gpu


def test_measured_rates_are_plausible():
    dfma, ms = h2.h2_measure_peak("dfma", 5.0)
    ffma, _ = h2.h2_measure_peak("ffma", 5.0)
    ex2, _ = h2.h2_measure_peak("ex2", 5.0)
    assert ms > 0.5
    # a GB300 runs FP64 FMAs at a few percent of its FP32 rate, and both far below 1e15/s
    assert 1e11 < dfma < ffma < 1e15
    assert 1e11 < ex2 < ffma


def test_measure_peak_rejects_bad_arguments():
    import ctypes as C
    lib = h2.load()
    r = C.c_double(0.0)
    assert lib.h2_measure_peak(7, 10.0, C.byref(r), None) == h2.H2_EINVAL
    assert lib.h2_measure_peak(0, 0.1, C.byref(r), None) == h2.H2_EINVAL
    assert lib.h2_measure_peak(0, 10.0, None, None) == h2.H2_EINVAL
