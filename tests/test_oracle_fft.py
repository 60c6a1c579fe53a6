"""Pins of the oracle's DFTs against numpy's FFT (an independent library) and
Parseval's theorem.  The forward sign is the paper's, exp(-2 pi j n k / N)
(Sec. 3.2, Eq. dft)."""
import numpy as np
import pytest

import oracle as orc


@pytest.mark.parametrize("log2n", list(range(0, 13)))
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_numpy(log2n, sign):
    n = 1 << log2n
    rng = np.random.default_rng(100 + log2n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x) if sign < 0 else n * np.fft.ifft(x)
    got = orc.fft(x, sign)
    scale = max(1.0, np.abs(ref).max())
    assert np.abs(got - ref).max() <= 1e-13 * scale * max(1, log2n)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 12, 64, 100])
def test_direct_dft_matches_numpy(n):
    rng = np.random.default_rng(7 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.abs(orc.dft(x, -1) - np.fft.fft(x)).max() <= 1e-12 * max(1, n)
    assert np.abs(orc.dft(x, +1) - n * np.fft.ifft(x)).max() <= 1e-12 * max(1, n)


def test_fft_matches_direct_dft_and_parseval():
    rng = np.random.default_rng(3)
    n = 512
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    X = orc.fft(x)
    assert np.abs(X - orc.dft(x)).max() < 1e-10
    assert abs(np.sum(np.abs(X) ** 2) / n - np.sum(np.abs(x) ** 2)) < 1e-9 * np.sum(np.abs(x) ** 2)


def test_fft_rejects_non_power_of_two():
    with pytest.raises(ValueError):
        orc.fft(np.ones(6, dtype=complex))


def test_fft_impulse_and_tone():
    n = 256
    d = np.zeros(n, complex)
    d[0] = 1.0
    assert np.allclose(orc.fft(d), np.ones(n), atol=1e-15)
    k0 = 17
    tone = np.exp(2j * np.pi * k0 * np.arange(n) / n)
    X = orc.fft(tone)
    expect = np.zeros(n, complex)
    expect[k0] = n
    assert np.abs(X - expect).max() < 1e-11
