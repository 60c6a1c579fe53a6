"""Pins of the oracle's two back-ends:

* Chirpolator: at DM = 0 the per-DM visibilities are the plain zero-lag
  correlator of the raw voltages (Sec. 2.4.3, FX correlation; p.q^* as in
  Eq. xpq); autocorrelations are real and non-negative; exchanging two antennas
  conjugates their visibility (V_qp = V_pq^*).
* Chimageator: at DM = 0 the beam powers are the plain phased-sum beamformer
  of the raw voltages (Sec. 2.4.2); a narrowband tone from direction (l, m)
  reaches beam amplitude M exactly at that pixel (the single-dump analogue of
  the ideal value of Eq. pthsum), and less elsewhere; the weights follow the
  geometric delay of Eq. tau3D (App. A.1).
* An injected pulse (sky model) reaches its analytic dump S/N.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1109_3186_gb300 import skymodel

C = 299792458.0


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def test_chirpolator_dm0_is_plain_correlator(k_dm):
    M, N, L = 4, 6000, 500
    x = _rand((M, N), 1)
    V = orc.chirpolator(x, 1.4e9, 8e6, k_dm, np.array([0.0]), 1024, L)[0]
    pairs = [(p, q) for p in range(M) for q in range(p, M)]
    for m in range(N // L):
        seg = x[:, m * L:(m + 1) * L]
        full = np.einsum("pt,qt->pq", seg, np.conj(seg))
        ref = np.array([full[p, q] for p, q in pairs])
        assert np.abs(V[m] - ref).max() < 1e-10 * np.abs(ref).max()


def test_visibility_symmetry(k_dm):
    M, N, L = 3, 30000, 1024
    x = _rand((M, N), 2)
    dms = np.array([0.0, 12.0, 40.0])
    V = orc.chirpolator(x, 1.4e9, 8e6, k_dm, dms, 4096, L)
    Vs = orc.chirpolator(x[[1, 0, 2]], 1.4e9, 8e6, k_dm, dms, 4096, L)
    # pair order (0,0) (0,1) (0,2) (1,1) (1,2) (2,2)
    assert np.abs(V[..., 1] - np.conj(Vs[..., 1])).max() < 1e-9
    autos = V[..., [0, 3, 5]]
    assert np.abs(autos.imag).max() < 1e-9
    assert (autos.real >= 0).all()
    assert np.abs(V[..., 0] - Vs[..., 3]).max() < 1e-9


def test_invalid_dumps_are_zero(k_dm):
    M, N, L = 2, 1 << 15, 1024
    x = _rand((M, N), 3)
    dms = np.array([0.0, 60.0])
    V = orc.chirpolator(x, 1.4e9, 8e6, k_dm, dms, 1 << 14, L)
    lay = orc.layout(dms, 1, 1.4e9, 8e6, k_dm, N, 1 << 14)
    first, last = orc.dump_range(N, lay["n_hi"], lay["n_lo"], L)
    assert first > 0 and last < N // L - 1
    assert np.all(V[1, :first] == 0) and np.all(V[1, last + 1:] == 0)
    assert np.all(np.abs(V[1, first:last + 1, 0]) > 0)
    assert np.all(np.abs(V[0, :, 0]) > 0)


def test_chimageator_dm0_is_plain_beamformer(k_dm):
    M, N, L = 5, 4096, 512
    x = _rand((M, N), 4)
    xyz = skymodel.antenna_positions(M, 3000.0, 5)
    pix = skymodel.pixel_grid(4, 1.0)
    P = orc.chimageator(x, 1.4e9, 8e6, k_dm, np.array([0.0]), 1024, L, xyz, pix)[0]
    W = orc.beam_weights(xyz, pix, 1.4e9)
    b = W @ x                                    # [n_pix, N]
    ref = (np.abs(b) ** 2).reshape(pix.shape[0], N // L, L).sum(-1).T
    assert np.abs(P - ref).max() < 1e-10 * ref.max()


def test_beam_weights_follow_tau3d():
    # antenna 1 on the u axis at 1500 m, antenna 2 raised by 10 m in w
    xyz = np.array([[0.0, 0.0, 0.0], [1500.0, 0.0, 0.0], [0.0, 0.0, 10.0]])
    th = math.radians(0.3)
    pix = np.array([[math.sin(th), 0.0], [0.0, math.sin(th)]])
    f0 = 1.4e9
    W = orc.beam_weights(xyz, pix, f0)
    assert abs(W[0, 0] - 1) < 1e-15
    ph = 2 * math.pi * f0 * 1500.0 * math.sin(th) / C        # b sin(theta)/c
    assert abs(W[0, 1] - complex(math.cos(ph), math.sin(ph))) < 1e-12
    assert abs(W[1, 1] - 1) < 1e-15
    ph_w = 2 * math.pi * f0 * 10.0 * (math.cos(th) - 1.0) / C  # w (sqrt(1-l^2-m^2)-1)/c
    assert abs(W[0, 2] - complex(math.cos(ph_w), math.sin(ph_w))) < 1e-12


def test_tone_from_direction_reaches_amplitude_m(k_dm):
    M, N, L = 7, 2048, 256
    xyz = skymodel.antenna_positions(M, 4000.0, 8)
    pix = skymodel.pixel_grid(5, 1.0)
    p0 = 7
    l0, m0 = pix[p0]
    f0, A = 1.4e9, 0.8
    tau = (xyz[:, 0] * l0 + xyz[:, 1] * m0 + xyz[:, 2] * (math.sqrt(1 - l0 * l0 - m0 * m0) - 1)) / C
    # a tone at the band centre (baseband f = 0) delayed by tau_a is the pure phase
    x = A * np.exp(-2j * math.pi * f0 * tau)[:, None] * np.ones((1, N))
    P = orc.chimageator(x, f0, 8e6, k_dm, np.array([0.0]), 1024, L, xyz, pix)[0]
    assert np.allclose(P[:, p0], (M * A) ** 2 * L, rtol=1e-12)
    others = np.delete(P, p0, axis=1)
    assert (others < P[:, [p0]] * (1 - 1e-6)).all()


@pytest.mark.slow
def test_injected_pulse_reaches_design_snr(k_dm):
    """Sky-model burst at boresight, true DM: the oracle's beam S/N in the
    pulse dump matches the sky model's analytic S/N (20) within the burst's
    own energy fluctuation and the noise."""
    sc = skymodel.chirpolator_small(n_samp=1 << 17, n_dm=5, dm_max=60.0, nfft_min=1 << 14,
                                    seed=1234)
    p = sc.pulses[0]
    p.l, p.m = 0.0, 0.0
    x = sc.voltages()
    d = int(np.argmin(np.abs(sc.dms - p.dm)))
    assert abs(sc.dms[d] - p.dm) < 1e-9
    m_p = int(p.t0 // sc.dump_len)
    pix = np.array([[0.0, 0.0]])
    P = orc.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len, sc.xyz, pix,
                        d_sel=[d], m0=m_p - 8, m1=m_p + 9)[0, :, 0]
    M, L = sc.n_ant, sc.dump_len
    snr = (P - M * L) / (M * math.sqrt(L))
    assert int(np.argmax(snr)) == 8
    assert 15.0 < snr[8] < 25.0
    assert np.abs(np.delete(snr, 8)).max() < 5.0
