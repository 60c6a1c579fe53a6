"""Pins of the oracle's dispersion sweep, chirp H_DM and overlap-save
dedispersion against what the paper fixes:

* Eq. 1 with mu ~ 4.15 ms GHz^2 (Sec. 2.1) and the Fig. 1 setting;
* |H_DM| = 1 and the group delay of H_DM undoing Eq. 1 about f0;
* the paper's analytic dispersed waveform (Eqs. freqvst and phit, Sec. 2.1)
  dedispersing to a single sample at its Eq. 1 arrival time at f0;
* DM = 0 reducing to the identity;
* the block grid checked against a brute-force circular convolution.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as orc

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_sweep_matches_eq1_with_paper_mu(k_dm):
    s = GOLD["fig_delayvsfreq_setting"]
    mu = GOLD["mu_ms_ghz2"]["value"]          # ms GHz^2
    f0, bw, dm = s["f0_mhz"] * 1e6, s["bw_mhz"] * 1e6, s["dm"]
    hi, lo = orc.sweep(f0, bw, k_dm, dm)
    f_hi, f_lo = (f0 + bw / 2) / 1e9, (f0 - bw / 2) / 1e9
    t_paper_ms = mu * dm * (f_lo ** -2 - f_hi ** -2)     # Eq. 1, t in ms
    t_oracle_ms = (hi + lo) / bw * 1e3
    # the paper prints mu to 3 significant figures
    assert abs(t_oracle_ms / t_paper_ms - 1.0) < 5e-3
    assert 125.0 < t_oracle_ms < 127.5
    # the upper half of the band sweeps faster than the lower half (nu^-2 law)
    t_hi_paper = mu * dm * ((f0 / 1e9) ** -2 - f_hi ** -2)
    assert abs(hi / bw * 1e3 / t_hi_paper - 1.0) < 5e-3
    assert lo > hi


def test_sweep_zero_dm_and_integer_ceiling(k_dm):
    assert orc.sweep(1.4e9, 8e6, k_dm, 0.0) == (0, 0)
    hi, lo = orc.sweep(1.4e9, 8e6, k_dm, 150.0)
    exact = k_dm * 150.0 * (1.4e9 ** -2 - (1.404e9) ** -2) * 8e6
    assert hi == math.ceil(exact)


@pytest.mark.parametrize("dm", [0.0, 3.0, 75.0, 2000.0])
def test_chirp_unit_modulus(k_dm, dm):
    H = orc.chirp(1.4e9, 8e6, k_dm, dm, 1 << 14)
    assert np.abs(np.abs(H) - 1.0).max() < 1e-14


def test_chirp_group_delay_undoes_eq1(k_dm):
    f0, bw, dm, n = 1.4e9, 8e6, 75.0, 1 << 16
    H = orc.chirp(f0, bw, k_dm, dm, n)
    fb = np.fft.fftfreq(n, d=1.0 / bw)
    order = np.argsort(fb)                 # ascending frequency, -B/2 .. B/2
    Hs, fs = H[order], fb[order]
    dphi = np.angle(Hs[1:] * np.conj(Hs[:-1]))
    df = bw / n
    tau_fd = -dphi / (2 * math.pi * df)    # group delay of H (s)
    f_mid = 0.5 * (fs[1:] + fs[:-1])
    # dedispersion must advance each frequency by the Eq. 1 lag relative to f0
    tau_eq1 = k_dm * dm * (1.0 / f0 ** 2 - 1.0 / (f0 + f_mid) ** 2)
    assert np.abs(tau_fd - tau_eq1).max() < 1e-9 * np.abs(tau_eq1).max() + 1e-12


def _analytic_dispersed_impulse(f0, bw, dm, n_samp, t_start, k_dm):
    """Baseband voltage of an impulse dispersed by Eq. 1, written in the time
    domain from the instantaneous frequency of Eq. freqvst and its integral,
    the phase of Eq. phit (exact form, not the Taylor truncation).  The
    amplitude nu^(3/2) makes the spectrum flat (stationary phase), so the
    undispersed signal is a delta.  Returns (s, arrival sample at f0)."""
    nu_top = f0 + bw / 2
    kd = k_dm * dm
    u = (np.arange(n_samp) - t_start) / bw
    T = kd * ((f0 - bw / 2) ** -2 - nu_top ** -2)
    inside = (u >= 0) & (u <= T)
    uu = np.where(inside, u, 0.0)
    root = np.sqrt(nu_top ** -2 + uu / kd)
    phase = 2 * math.pi * (2 * kd * (root - 1.0 / nu_top) - f0 * uu)
    s = np.where(inside, root ** -1.5, 0.0) * np.exp(1j * phase)
    return s, t_start + kd * (f0 ** -2 - nu_top ** -2) * bw


@pytest.mark.parametrize("f0,bw,dm,n_samp,nfft", [
    (1.4e9, 8e6, 75.0, 1 << 17, 1 << 16),
    (1.4e9, 8e6, 150.0, 1 << 17, 1 << 16),
    (1.4e9, 32e6, 40.0, 1 << 19, 1 << 18),
    (1.4e9, 8e6, 10.0, 1 << 15, 1 << 14),
])
def test_dispersed_impulse_dedisperses_to_delta(k_dm, f0, bw, dm, n_samp, nfft):
    s, t_f0 = _analytic_dispersed_impulse(f0, bw, dm, n_samp, 20000.0, k_dm)
    # shift the start so that the arrival at f0 falls on a sample
    s, t_f0 = _analytic_dispersed_impulse(f0, bw, dm, n_samp, 20000.0 + round(t_f0) - t_f0, k_dm)
    y = orc.dedisperse(s[None, :], f0, bw, k_dm, np.array([dm]), 0, nfft)[0]
    e = np.abs(y) ** 2
    c = int(round(t_f0))
    assert int(np.argmax(e)) == c
    assert e[c] / e.sum() > 0.985
    assert e[c - 2:c + 3].sum() / e.sum() > 0.985


def test_dm_zero_is_identity(k_dm):
    rng = np.random.default_rng(5)
    x = rng.standard_normal((3, 5000)) + 1j * rng.standard_normal((3, 5000))
    y = orc.dedisperse(x, 1.4e9, 8e6, k_dm, np.array([0.0, 20.0]), 0, 1024)
    assert np.abs(y - x).max() < 1e-12


def _owner(t, n_hi_max, step, n_blk):
    if n_blk <= 1:
        return 0
    return min(max((t - n_hi_max) // step, 0), n_blk - 1)


def test_blocks_match_bruteforce_circular_convolution(k_dm):
    f0, bw, n_samp, nfft_min = 1.4e9, 8e6, 3000, 512
    dms = np.array([0.0, 2.0, 4.0, 6.0])
    rng = np.random.default_rng(11)
    x = rng.standard_normal(n_samp) + 1j * rng.standard_normal(n_samp)
    for d in range(len(dms)):
        lay = orc.layout(dms, d, f0, bw, k_dm, n_samp, nfft_min)
        nfft, step = lay["nfft"], lay["step"]
        y = orc.dedisperse(x[None, :], f0, bw, k_dm, dms, d, nfft_min)[0]
        h = np.fft.ifft(orc.chirp(f0, bw, k_dm, dms[d], nfft))   # impulse response
        idx = np.arange(nfft)
        for t in range(n_samp):
            valid = lay["n_hi"] <= t < n_samp - lay["n_lo"]
            if not valid:
                assert y[t] == 0
                continue
            b = _owner(t, lay["n_hi_max"], step, lay["n_blk"])
            s0 = b * step
            blk = np.zeros(nfft, complex)
            seg = x[s0:s0 + nfft]
            blk[:seg.size] = seg
            i = t - s0
            assert lay["n_hi"] <= i < nfft - lay["n_lo"]
            ref = np.sum(blk * h[(i - idx) % nfft])
            assert abs(y[t] - ref) < 1e-10


def test_valid_outputs_approximate_linear_convolution(k_dm):
    """Overlap-save keeps only outputs whose support lies inside the block: they
    must agree (to the chirp's band-edge tail level) with one long transform
    over the whole series.  Discarding the wrong ends gives O(1) errors."""
    f0, bw, n_samp = 1.4e9, 8e6, 1 << 16
    dms = np.array([30.0])
    rng = np.random.default_rng(2)
    x = rng.standard_normal(n_samp) + 1j * rng.standard_normal(n_samp)
    y_blk = orc.dedisperse(x[None, :], f0, bw, k_dm, dms, 0, 1 << 13)[0]
    y_long = orc.dedisperse(x[None, :], f0, bw, k_dm, dms, 0, 1 << 18)[0]
    lay = orc.layout(dms, 0, f0, bw, k_dm, n_samp, 1 << 13)
    assert lay["n_blk"] > 4
    v = slice(lay["n_hi"], n_samp - lay["n_lo"])
    err = np.sqrt(np.mean(np.abs(y_blk[v] - y_long[v]) ** 2) / np.mean(np.abs(y_long[v]) ** 2))
    assert err < 0.05


def test_span_is_slice_of_full(k_dm):
    rng = np.random.default_rng(9)
    x = rng.standard_normal((2, 20000)) + 1j * rng.standard_normal((2, 20000))
    dms = np.array([0.0, 10.0, 25.0])
    full = orc.dedisperse(x, 1.4e9, 8e6, k_dm, dms, 2, 2048)
    part = orc.dedisperse(x, 1.4e9, 8e6, k_dm, dms, 2, 2048, 7000, 13000)
    assert np.array_equal(part, full[:, 7000:13000])


def test_layout_groups_follow_the_fft_length_rule(k_dm):
    # 6 antennas, 8 MHz at 1.4 GHz, 2^20 samples, 16 DMs in 0-150, FFT 2^16
    dms = np.linspace(0, 150, 16)
    lay = orc.layout(dms, 15, 1.4e9, 8e6, k_dm, 1 << 20, 1 << 16)
    assert lay["nfft"] == 1 << 16
    assert lay["step"] == ((1 << 16) - lay["n_hi"] - lay["n_lo"]) // 8 * 8
    assert lay["n_blk"] == 28
    # 12 antennas, 32 MHz, 2^22 samples, 64 DMs in 0-300, FFT >= 2^18
    dms = np.linspace(0, 300, 64)
    sizes = [orc.layout(dms, d, 1.4e9, 32e6, k_dm, 1 << 22, 1 << 18)["nfft"] for d in range(64)]
    counts = {n: sizes.count(n) for n in sorted(set(sizes))}
    assert counts == {1 << 18: 9, 1 << 19: 9, 1 << 20: 18, 1 << 21: 28}
    for d in range(64):
        lay = orc.layout(dms, d, 1.4e9, 32e6, k_dm, 1 << 22, 1 << 18)
        assert lay["nfft"] >= 2 * (lay["n_hi_max"] + lay["n_lo_max"])   # >= 50 % kept


@pytest.mark.parametrize("dm", [0.0, 3.7, 48.0, 150.0])
def test_whole_block_products_do_not_depend_on_dm(k_dm, dm):
    """Unitarity: over one whole circular block, dedispersion (forward FFT,
    chirp multiply, inverse FFT with 1/N) leaves every antenna-pair product
    sum unchanged, sum_t y_p y_q^* = sum_t x_p x_q^* for any DM, because
    |H| = 1 (Parseval on both sides).  A chirp with the wrong modulus, a
    missing or doubled 1/N, or a chirp applied to one antenna only fails."""
    nfft = 1 << 12
    rng = np.random.default_rng(5)
    x = (rng.standard_normal((3, nfft)) + 1j * rng.standard_normal((3, nfft))) / math.sqrt(2)
    H = orc.chirp(1.4e9, 8e6, k_dm, dm, nfft)
    y = np.array([orc.fft(orc.fft(x[a]) * H, +1) / nfft for a in range(3)])
    G_x = x @ x.conj().T
    G_y = y @ y.conj().T
    assert np.abs(G_y - G_x).max() <= 1e-9 * np.abs(G_x).max()
    if dm > 0:
        # the voltages themselves do change (the products would not pin anything otherwise)
        assert np.abs(y - x).max() > 0.1
