"""True-delay (wideband) beams on the GPU (chirp_truedelay_run) against the
FP64 oracle (oracle/truedelay.py: per overlap-save block and frequency bin
the antenna spectra weighted by exp(+2 pi j (f0 + f) tau_a), Eq. tau3D,
times the chirp; inverse transform over the owned samples; |.|^2 summed per
dump).

Checked:
- element by element against the oracle on seeded noise plus a burst, for a
  6 km array at 32 MHz (B tau up to several samples) and 25 pixels (two
  pixel chunks per thread block), three DMs in three FFT-length groups,
  within the FP32 path's 1e-5 relative;
- with every antenna at the origin the true-delay beams are the phased beams
  of chimageator_run (same search, FP32 tolerance);
- a noise-free burst from a pixel's direction reaches M^2 times one origin
  antenna's power there (the oracle's pin, now through the GPU), while the
  narrowband phased beam of the same plan loses over 10 % to smearing.
"""
import numpy as np
import pytest

import oracle
import paper_1109_3186_gb300 as chirp
from oracle import truedelay
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_POW, pow_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K_DM = skymodel.K_DM
F0, BW, L, NMIN = 1.4e9, 32e6, 1024, 1 << 13


def _run(x, xyz, pix, dms, n_samp, beam_mode=chirp.BEAM_AUTO):
    plan = chirp.Plan(xyz, F0, BW, n_samp, dms, L, NMIN, pix_lm=pix, k_dm=K_DM,
                      beam_mode=beam_mode)
    P = torch.full((len(dms), plan.n_dump, plan.n_pix), -1.0, dtype=torch.float32, device="cuda")
    plan.truedelay(torch.from_numpy(x).cuda(), P)
    Pb = torch.empty_like(P)
    plan.chimageator(torch.from_numpy(x).cuda(), Pb)
    torch.cuda.synchronize()
    plan.close()
    return P.cpu().numpy(), Pb.cpu().numpy()


def test_truedelay_beams_match_the_oracle():
    n_samp = 1 << 16
    xyz = skymodel.antenna_positions(6, 6000.0, 31)
    pix = skymodel.pixel_grid(5, 1.0)
    dms = np.array([0.0, 3.0, 12.0])
    x = skymodel.noise(6, n_samp, 32)
    p = skymodel.Pulse(dm=3.0, t0=40.5 * L, fwhm_s=20e-6,
                       amp=skymodel.burst_amplitude(30.0, 6, L, 20e-6 * BW, L / 2),
                       l=pix[7][0], m=pix[7][1], seed=33)
    skymodel.inject(x, xyz, F0, BW, p)
    P, _ = _run(x, xyz, pix, dms, n_samp)
    Po = truedelay.beams(x, xyz, pix, F0, BW, K_DM, dms, NMIN, L)
    assert len({oracle.layout(dms, d, F0, BW, K_DM, n_samp, NMIN)["nfft"] for d in range(3)}) >= 2
    assert np.array_equal(P == 0, Po == 0)
    err = pow_error(P, Po)
    assert err <= TOL_POW, err
    assert int(np.argmax(P[1, 40])) == 7


def test_antennas_at_the_origin_give_the_phased_beams():
    n_samp = 1 << 15
    xyz = np.zeros((4, 3))
    pix = np.array([[0.0, 0.0], [0.004, -0.002], [-0.003, 0.001]])
    dms = np.array([0.0, 1.5])
    x = skymodel.noise(4, n_samp, 3)
    P, Pb = _run(x, xyz, pix, dms, n_samp, beam_mode=chirp.BEAM_FP32_SIMT)
    assert np.array_equal(P == 0, Pb == 0)
    assert pow_error(P, Pb.astype(np.float64)) <= TOL_POW


def _burst(xyz, l, m, n_samp, dm):
    """A noise-free dispersed burst as received by antennas xyz from (l, m),
    delayed exactly on the n_samp-point grid (the search's single block)."""
    s = np.zeros((1, n_samp), np.complex64)
    p = skymodel.Pulse(dm=dm, t0=0.55 * n_samp, fwhm_s=2e-6, amp=1.0, l=0.0, m=0.0, seed=9)
    skymodel.inject(s, np.zeros((1, 3)), F0, BW, p)
    S = np.fft.fft(s[0].astype(np.complex128))
    b = np.arange(n_samp)
    f = np.where(b < n_samp // 2, b, b - n_samp) * BW / n_samp
    tau = skymodel.geometric_delay(np.asarray(xyz), l, m)
    return np.stack([np.fft.ifft(S * np.exp(-2j * np.pi * (F0 + f) * t)) for t in tau])


def test_a_burst_from_the_pixel_adds_coherently_at_every_frequency():
    n_samp, dm = 1 << 14, 2.0
    xyz = skymodel.antenna_positions(5, 6000.0, 11)
    l, m = 0.02, -0.012
    dms = np.array([dm])
    pix = np.array([[l, m]])
    x = _burst(xyz, l, m, n_samp, dm).astype(np.complex64)
    P, Pn = _run(x, xyz, pix, dms, n_samp, beam_mode=chirp.BEAM_FP32_SIMT)
    one = oracle.chimageator(_burst(np.zeros((1, 3)), l, m, n_samp, dm), F0, BW, K_DM, dms, NMIN,
                             L, np.zeros((1, 3)), pix)
    big = one > 1e-3 * one.max()
    assert (np.abs(P[big] - 25.0 * one[big]) / (25.0 * one[big])).max() <= 1e-4
    assert Pn.max() < 0.9 * P.max()
