"""Pins of the true-delay beam oracle (oracle/truedelay.py): with every
antenna at the origin it is the C oracle's phased beam; a noise-free burst
from a pixel's direction (the sky model applies the exact RF delay) gives
exactly M^2 times the power one antenna at the origin would see, while the
narrowband phased beam loses power to bandwidth smearing; a planted sign
error in the delays fails."""
import numpy as np

import oracle
from oracle import truedelay
from paper_1109_3186_gb300 import skymodel

K_DM = skymodel.K_DM
F0, BW, L, NMIN = 1.4e9, 32e6, 1024, 1 << 12


def test_antennas_at_the_origin_give_the_phased_beam():
    x = skymodel.noise(4, 1 << 14, 3)
    xyz = np.zeros((4, 3))
    pix = np.array([[0.0, 0.0], [0.004, -0.002]])
    dms = np.array([0.0, 1.5])
    P = truedelay.beams(x, xyz, pix, F0, BW, K_DM, dms, NMIN, L)
    Po = oracle.chimageator(x, F0, BW, K_DM, dms, NMIN, L, xyz, pix)
    assert np.abs(P - Po).max() <= 1e-9 * Po.max()


def _burst(xyz, l, m, n_samp, dm):
    """A noise-free dispersed burst as received by antennas xyz from (l, m):
    the origin's signal s (sky model, one antenna at the origin), delayed
    per antenna by exp(-2 pi j (f0 + f) tau_a) on the n_samp-point grid that
    is also the search's single overlap-save block (so the delay is exact)."""
    s = np.zeros((1, n_samp), np.complex64)
    p = skymodel.Pulse(dm=dm, t0=0.55 * n_samp, fwhm_s=2e-6, amp=1.0, l=0.0, m=0.0, seed=9)
    skymodel.inject(s, np.zeros((1, 3)), F0, BW, p)
    S = np.fft.fft(s[0].astype(np.complex128))
    b = np.arange(n_samp)
    f = np.where(b < n_samp // 2, b, b - n_samp) * BW / n_samp
    tau = np.array([skymodel.geometric_delay(np.asarray(xyz)[a:a + 1], l, m)[0] for a in range(len(xyz))])
    return np.stack([np.fft.ifft(S * np.exp(-2j * np.pi * (F0 + f) * t)) for t in tau]).astype(np.complex128)


def _aligned_ok():
    n_samp, dm = 1 << 14, 2.0
    xyz = skymodel.antenna_positions(5, 6000.0, 11)
    l, m = 0.02, -0.012
    dms = np.array([dm])
    P = truedelay.beams(_burst(xyz, l, m, n_samp, dm), xyz, np.array([[l, m]]), F0, BW, K_DM,
                        dms, NMIN, L)
    one = oracle.chimageator(_burst(np.zeros((1, 3)), l, m, n_samp, dm), F0, BW, K_DM, dms, NMIN,
                             L, np.zeros((1, 3)), np.array([[l, m]]))
    ok = np.abs(P - 25.0 * one).max() <= 1e-9 * (25.0 * one).max()
    return ok, P, xyz, l, m, dms, n_samp, dm


def test_a_burst_from_the_pixel_adds_coherently_at_every_frequency():
    ok, P, xyz, l, m, dms, n_samp, dm = _aligned_ok()
    assert ok and P.max() > 0
    # the narrowband phased beam at the same pixel loses power (B tau of a few samples here)
    Pn = oracle.chimageator(_burst(xyz, l, m, n_samp, dm), F0, BW, K_DM, dms, NMIN, L, xyz,
                            np.array([[l, m]]))
    assert Pn.max() < 0.9 * P.max()


def test_planted_sign_error_in_the_delays_fails(monkeypatch):
    good = truedelay._delays
    monkeypatch.setattr(truedelay, "_delays", lambda xyz, l, m: -good(xyz, l, m))
    ok, *_ = _aligned_ok()
    assert not ok
