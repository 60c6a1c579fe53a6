"""Pins of the oracle's incoherent path (Sec. 2.3.1 incoherent dedispersion of
the power beam, Sec. 2.4.1): the filterbank against closed forms (a tone at a
channel centre lands in that channel only, with the power the DFT gives;
Parseval over each block), and the shift-and-sum against the Eq. dmdelay
delays (a spectrogram holding one spike per channel at the Eq. dmdelay lag
adds up in a single output sample; DM = 0 is the plain channel sum)."""
import math

import numpy as np
import pytest

import oracle as orc


def test_tone_at_channel_centre(k_dm):
    n_chan, n_int, M, bw, f0 = 32, 4, 3, 8e6, 1.4e9
    N = n_chan * n_int * 5
    c0 = 21
    f_off = (c0 - n_chan // 2) * bw / n_chan            # channel centre offset
    A = 0.7
    t = np.arange(N)
    x = np.tile(A * np.exp(2j * math.pi * f_off * t / bw), (M, 1))
    S = orc.filterbank(x, n_chan, n_int)
    expect = M * n_int * (n_chan * A) ** 2
    assert np.allclose(S[c0], expect, rtol=1e-12)
    assert np.abs(np.delete(S, c0, axis=0)).max() < 1e-12 * expect


def test_filterbank_parseval_and_order():
    rng = np.random.default_rng(4)
    n_chan, n_int, M = 16, 8, 2
    x = rng.standard_normal((M, n_chan * n_int * 7)) + 1j * rng.standard_normal((M, n_chan * n_int * 7))
    S = orc.filterbank(x, n_chan, n_int)
    blocks = (np.abs(x) ** 2).reshape(M, 7, n_int * n_chan).sum(axis=(0, 2))
    assert np.allclose(S.sum(0), n_chan * blocks, rtol=1e-12)
    # numpy's FFT with fftshift gives the same channel order
    X = np.fft.fftshift(np.fft.fft(x.reshape(M, -1, n_chan), axis=-1), axes=-1)
    ref = (np.abs(X) ** 2).sum(0).reshape(7, n_int, n_chan).sum(1).T
    assert np.allclose(S, ref, rtol=1e-10)


def test_channel_shift_follows_eq1(k_dm):
    f0, bw, n_chan, n_int, dm = 1.4e9, 32e6, 32, 64, 150.0
    t_fb = n_chan * n_int / bw
    for c in (0, 7, 16, 31):
        fc = f0 + (c - n_chan // 2) * bw / n_chan
        lag = k_dm * dm * (fc ** -2 - f0 ** -2)          # Eq. dmdelay relative to f0
        assert orc.channel_shift(f0, bw, k_dm, dm, n_chan, n_int, c) == math.floor(lag / t_fb + 0.5)
    assert orc.channel_shift(f0, bw, k_dm, dm, n_chan, n_int, n_chan // 2) == 0
    assert orc.channel_shift(f0, bw, k_dm, dm, n_chan, n_int, 0) > 0      # low band later
    assert orc.channel_shift(f0, bw, k_dm, dm, n_chan, n_int, n_chan - 1) < 0


def test_dispersed_spikes_add_up(k_dm):
    f0, bw, n_chan, n_int = 1.4e9, 32e6, 32, 64
    T = 600
    dms = np.array([0.0, 80.0, 160.0])
    t0 = 300
    S = np.zeros((n_chan, T))
    for c in range(n_chan):
        S[c, t0 + orc.channel_shift(f0, bw, k_dm, 160.0, n_chan, n_int, c)] = 1.0 + c
    D = orc.incoherent(S, f0, bw, k_dm, n_int, dms)
    assert D[2, t0] == pytest.approx(sum(1.0 + c for c in range(n_chan)))
    assert D[2].argmax() == t0
    assert D[1].max() < D[2, t0]
    # DM 0: the plain channel sum
    assert np.allclose(D[0], S.sum(0))
