"""Pins of the Chirpolator pre-integrator oracle (oracle/cpi.py) against what
the paper and the mathematics fix, independent of the oracle's own formulas:
the Dirichlet response of a tone (Eq. phidn), the mixing tone of two
delayed linear chirps at k_0 = B tau (Eqs. xpq, f0Bt), the moving sum against
a brute-force windowed DFT (Eq. block_cic), the DFT factorisation across
window lengths (Sec. A.3.3), the closed-form image of a perfect chirp
(Eqs. pth, eth), and the paper's printed numbers (delta_mix ~ 7, FWHM 0.844)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import cpi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
K_DM = 4.148808e15


def _brute_window_dft(x, n0, N, ks):
    """sum_{n<N} exp(-2 pi j n k / N) x[n0 + n] by an explicit loop over k."""
    n = np.arange(N)
    return np.array([np.sum(np.exp(-2j * math.pi * n * k / N) * x[n0:n0 + N]) for k in ks])


def test_dirichlet_is_the_geometric_sum():
    for N in (8, 100, 4096):
        for x in (0.0, 0.3, 1.0, -2.5, 7.25):
            geo = abs(np.sum(np.exp(2j * math.pi * np.arange(N) * x / N)))
            assert abs(abs(cpi.dirichlet(x, N)) - geo) < 1e-9 * N


def test_tone_through_partial_dfts_and_moving_sum_is_phi_times_dirichlet():
    # a tone of kappa bins over an N-sample window (Eq. phidn)
    L, nw, K = 64, 6, 5
    N = L * nw
    kap = 2.37
    n = np.arange(3 * N)
    x = np.exp(2j * math.pi * kap * n / N)[None, :]
    X = cpi.window_local(cpi.cic(cpi.partial_dft(x, L, N, K), nw), nw, K)
    for m in (nw - 1, nw + 3, 2 * nw + 1):
        n0 = (m + 1 - nw) * L
        for k in range(-K, K + 1):
            want = (np.exp(2j * math.pi * kap * n0 / N) * np.exp(-1j * math.pi * (k - kap) * (N - 1) / N)
                    * (math.sin(math.pi * (k - kap)) / math.sin(math.pi * (k - kap) / N)))
            assert abs(X[k + K, m, 0] - want) < 1e-9 * N


def test_moving_sum_equals_brute_force_windowed_dft():
    rng = np.random.default_rng(5)
    L, nw, K = 32, 5, 4
    N = L * nw
    x = (rng.standard_normal((2, 20 * L)) + 1j * rng.standard_normal((2, 20 * L)))
    X = cpi.window_local(cpi.cic(cpi.partial_dft(x, L, N, K), nw), nw, K)
    for m in (nw - 1, 9, 19):
        for c in range(2):
            want = _brute_window_dft(x[c], (m + 1 - nw) * L, N, range(-K, K + 1))
            assert np.abs(X[:, m, c] - want).max() < 1e-9 * np.abs(want).max()
    assert np.all(X[:, :nw - 1] == 0)


def test_factorised_dft_is_a_sum_of_shorter_windows():
    # Sec. A.3.3: bin k of the n_win-block window = sum of D adjacent windows of
    # n_win / D blocks at bin k / D (absolute phases, before the window shift)
    rng = np.random.default_rng(8)
    L, nw, D = 16, 6, 3
    x = rng.standard_normal((1, 30 * L)) + 1j * rng.standard_normal((1, 30 * L))
    S_long = cpi.cic(cpi.partial_dft(x, L, nw * L, 6), nw)
    S_short = cpi.cic(cpi.partial_dft(x, L, nw // D * L, 2), nw // D)
    for k in (-6, -3, 3, 6):
        for m in (nw + 2, 25):
            want = sum(S_short[k // D + 2, m - i * (nw // D), 0] for i in range(D))
            assert abs(S_long[k + 6, m, 0] - want) < 1e-9 * abs(want)


def test_two_delayed_linear_chirps_mix_to_a_tone_at_b_tau():
    # Sec. 3.2: s(t) = exp(pi j fdot t^2), fdot = -B/T; antenna q sees s(t - tau)
    B, T = 4e6, 2e-3
    N = int(B * T)
    fdot = -B / T
    t = np.arange(N) / B
    for tau in (0.9e-6, -1.6e-6, 2.3e-6):
        y = np.stack([np.exp(1j * math.pi * fdot * t ** 2), np.exp(1j * math.pi * fdot * (t - tau) ** 2)])
        x = cpi.mix(y)
        L = N // 8
        K = 16
        X = cpi.window_local(cpi.cic(cpi.partial_dft(x, L, N, K), 8), 8, K)[:, 7, 0]
        k0 = fdot * tau * N / B                    # Eq. f0Bt with the chirp's sign: -B tau
        assert abs(k0 + B * tau) < 1e-9
        peak = int(np.argmax(np.abs(X))) - K
        assert abs(peak - k0) <= 0.5
        # Eq. phidn with Eq. phipq1: X_k = exp(-pi j fdot tau^2) exp(-pi j x (N-1)/N) D_N(x), x = k - k0
        for k in range(peak - 2, peak + 3):
            xk = k - k0
            want = (np.exp(-1j * math.pi * fdot * tau ** 2) * np.exp(-1j * math.pi * xk * (N - 1) / N)
                    * math.sin(math.pi * xk) / math.sin(math.pi * xk / N))
            assert abs(X[k + K] - want) < 1e-6 * N


def _model_voltages(xyz, l, m, f0, bw, dm, L, m_win, n_samp):
    """Baseband voltages of a unit linear chirp (rate a1, centre a0 at the
    midpoint of window m_win) from direction (l, m): y_a(t) = s(t - tau_a)
    exp(-2 pi j f0 tau_a) with s(t) = exp(2 pi j ((a0 - f0)(t - tc) + fdot (t - tc)^2 / 2))."""
    _, a0, a1 = cpi.chirp_model(f0, bw, K_DM, dm)
    nw = cpi.window_blocks(f0, bw, K_DM, dm, L)
    tc = ((m_win + 1 - nw) * L + nw * L / 2) / bw
    t = np.arange(n_samp) / bw
    tau = cpi.delays(xyz, [(l, m)])[0]
    y = np.empty((len(xyz), n_samp), np.complex128)
    for a in range(len(xyz)):
        u = t - tc - tau[a]
        y[a] = np.exp(2j * math.pi * ((a0 - f0) * u + 0.5 * a1 * u * u)) * np.exp(-2j * math.pi * f0 * tau[a])
    return y, nw


def test_image_of_a_perfect_chirp_is_the_closed_form_and_peaks_at_its_pixel():
    f0, bw, dm, L, F = 1.4e9, 8e6, 40.0, 64, 2
    rng = np.random.default_rng(4)
    xyz = np.zeros((5, 3))
    xyz[:, :2] = rng.uniform(-3000, 3000, (5, 2))
    xyz[:, 2] = rng.uniform(-20, 20, 5)
    ang = np.radians(np.linspace(-0.6, 0.6, 7))
    pix = np.array([(math.sin(a), math.sin(b)) for b in ang for a in ang])
    true = 17
    nw = cpi.window_blocks(f0, bw, K_DM, dm, L)
    m_win = nw + 4
    y, _ = _model_voltages(xyz, *pix[true], f0, bw, dm, L, m_win, (m_win + 3) * L)
    E, kept, K = cpi.search(y, xyz, pix, f0, bw, K_DM, [dm], L, F, keep=True)
    # closed form: P = sum_pq sum_k D_N(k - kappa)^2 / N
    _, a0, a1 = cpi.chirp_model(f0, bw, K_DM, dm)
    N = nw * L
    tau = cpi.delays(xyz, pix[true:true + 1])[0]
    P = 0.0
    for p, q in cpi.pairs(5):
        kap = -a1 * (tau[p] - tau[q]) * N / bw
        ks = np.arange(int(np.rint(kap)) - F, int(np.rint(kap)) + F + 1)
        P += float(np.sum(cpi.dirichlet(ks - kap, N) ** 2)) / N
    assert abs(E[0, m_win, true] - P * P) < 1e-9 * P * P
    assert int(np.argmax(E[0, m_win])) == true
    assert np.all(E[0, :nw - 1] == 0)


def test_gauss_sum_fixed_values():
    # Eq. gaussum: G(0, L) = L, |G(a, L)| < L otherwise; G(1/2, L) alternates
    assert cpi.gauss_sum(0.0, 1000) == pytest.approx(1000.0)
    assert abs(cpi.gauss_sum(1e-5, 1000)) < 1000.0
    assert cpi.gauss_sum(0.5, 10) == pytest.approx(0.0, abs=1e-9)   # sum of (-1)^(n^2) = (-1)^n
    assert cpi.gauss_sum(0.5, 11) == pytest.approx(1.0, abs=1e-9)


def test_paper_numbers_delta_mix_and_resolution():
    g = json.load(open(GOLDEN))
    ex = g["delta_mix_example"]
    tau = ex["baseline_m"] * math.sin(math.radians(ex["theta_deg"])) / 299792458.0
    dmx = cpi.delta_mix(ex["f_centre_hz"], ex["bandwidth_hz"], K_DM, ex["dm"], tau)
    assert round(dmx) == ex["delta_mix_bins"]
    # D_N^2 full width at half maximum: exact sinc^2 width 0.8859 bins; the
    # paper's third-order Taylor estimate (Eq. fwhm) is 0.844
    w = cpi.fwhm_bins()
    assert abs(w - 2 * 0.442946470) < 1e-6
    taylor = 2.0 / math.pi * math.sqrt(6 * (1 - 1 / math.sqrt(2)))
    assert round(taylor, 3) == g["chirpolator_fwhm_bins"]


def test_chirp_model_rate_and_window():
    # a1 ~ -B/T (Sec. 2.1); the mean slope differs from the midpoint slope by
    # the band's curvature: ~5 % at 400 MHz, ~1e-4 at 32 MHz around 1.4 GHz
    for bw, tol in ((400e6, 0.06), (32e6, 1e-3)):
        T, a0, a1 = cpi.chirp_model(1.4e9, bw, K_DM, 100.0)
        assert abs(a1 / (-bw / T) - 1) < tol
        assert 1.4e9 - bw / 2 < a0 < 1.4e9
    T, _, _ = cpi.chirp_model(1.4e9, 400e6, K_DM, 100.0)
    assert abs(T - 0.1261) < 5e-4                     # the 126 ms of Fig. delayvsfreq
    assert cpi.window_blocks(1.4e9, 32e6, K_DM, 300.0, 2048) == 454
    with pytest.raises(ValueError):
        cpi.chirp_model(1.4e9, 32e6, K_DM, 0.0)


def _two_chirp_peak_ok() -> bool:
    B, T = 4e6, 2e-3
    N = int(B * T)
    fdot = -B / T
    t = np.arange(N) / B
    tau = 1.6e-6
    y = np.stack([np.exp(1j * math.pi * fdot * t ** 2), np.exp(1j * math.pi * fdot * (t - tau) ** 2)])
    X = cpi.window_local(cpi.cic(cpi.partial_dft(cpi.mix(y), N // 8, N, 16), 8), 8, 16)[:, 7, 0]
    return abs(int(np.argmax(np.abs(X))) - 16 - fdot * tau * N / B) <= 0.5


def _perfect_chirp_ok() -> bool:
    f0, bw, dm, L, F = 1.4e9, 8e6, 40.0, 64, 1
    xyz = np.array([[0.0, 0, 0], [2500.0, 300, 0], [-700.0, 2100, 0]])
    pix = np.array([(0.004, -0.003), (0.0, 0.0)])
    nw = cpi.window_blocks(f0, bw, K_DM, dm, L)
    y, _ = _model_voltages(xyz, *pix[0], f0, bw, dm, L, nw, (nw + 2) * L)
    E = cpi.search(y, xyz, pix, f0, bw, K_DM, [dm], L, F)
    _, _, a1 = cpi.chirp_model(f0, bw, K_DM, dm)
    tau = cpi.delays(xyz, pix[:1])[0]
    P = 0.0
    for p, q in cpi.pairs(3):
        kap = -a1 * (tau[p] - tau[q]) * nw * L / bw
        ks = np.arange(int(np.rint(kap)) - F, int(np.rint(kap)) + F + 1)
        P += float(np.sum(cpi.dirichlet(ks - kap, nw * L) ** 2)) / (nw * L)
    return abs(E[0, nw, 0] - P * P) < 1e-9 * P * P


def test_planted_mistakes_fail_a_pin(monkeypatch):
    """Mistakes planted in the oracle (each undone after its check) are caught:
    a conjugated mixing product, a wrong sign of the window shift, a dropped
    fringe term in the filter, and a moving sum one block too long."""
    assert _two_chirp_peak_ok() and _perfect_chirp_ok()
    good_mix, good_win, good_w, good_cic = cpi.mix, cpi.window_local, cpi.image_weights, cpi.cic
    monkeypatch.setattr(cpi, "mix", lambda y: np.conj(good_mix(y)))
    assert not _two_chirp_peak_ok()
    monkeypatch.setattr(cpi, "mix", good_mix)

    def win_bad(S, n_win, K):
        return np.conj(good_win(np.conj(S), n_win, K))
    monkeypatch.setattr(cpi, "window_local", win_bad)
    assert not _perfect_chirp_ok()
    monkeypatch.setattr(cpi, "window_local", good_win)

    def w_bad(xyz, pix_lm, f0, bw, k_dm, dm, blk_len, F):
        k0p, W = good_w(xyz, pix_lm, f0 + 1e5, bw, k_dm, dm, blk_len, F)
        return k0p, W
    monkeypatch.setattr(cpi, "image_weights", w_bad)
    assert not _perfect_chirp_ok()
    monkeypatch.setattr(cpi, "image_weights", good_w)

    monkeypatch.setattr(cpi, "cic", lambda V, n_win: good_cic(V, n_win + 1))
    assert not _perfect_chirp_ok()
