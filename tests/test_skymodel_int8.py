"""The int8 input generator: per-component RMS of 16 counts, rounding to the
nearest code (numpy's rint, ties to even), clamp at +-127, and the FP32
dequantisation the int8 ingest performs."""
import numpy as np

from paper_1109_3186_gb300 import skymodel


def test_quantiser_rms_rounding_and_clamp():
    x = skymodel.noise(3, 1 << 16, 5)
    x[1, 100] = 100.0 + 0j                   # far outside the range: clamped
    q, s = skymodel.quantize_ci8(x)
    assert q.dtype == np.int8 and q.shape == (3, 1 << 16, 2)
    rms = np.sqrt((q.astype(np.float64) ** 2).mean(axis=(1, 2)))
    assert np.all(np.abs(rms[[0, 2]] - 16.0) < 0.2)   # antenna 1 lost power to the clamp
    assert q[1, 100, 0] == 127 and q[1, 100, 1] == 0
    g = 1.0 / s.astype(np.float64)
    # away from the clamp the code is the nearest integer to x * gain
    r = x[0, :1000].real * g[0]
    assert np.all(np.abs(q[0, :1000, 0] - r) <= 0.5 + 1e-6)


def test_dequantisation_is_scale_times_code_in_fp32():
    q = np.array([[[3, -4], [127, -127]]], np.int8)
    s = np.array([0.1], np.float32)
    y = skymodel.dequantize_ci8(q, s)
    assert y.dtype == np.complex64
    assert y[0, 0] == np.complex64(np.float32(3) * np.float32(0.1) + 1j * (np.float32(-4) * np.float32(0.1)))
    assert y[0, 1].real == np.float32(127) * np.float32(0.1)
