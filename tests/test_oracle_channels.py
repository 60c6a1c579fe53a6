"""Pins of the coarse-channel combination oracle (oracle/channels.py): DM 0
is a plain sum, the alignment shifts follow Eq. dmdelay through the C
oracle's independently pinned sweep, and a burst injected into each
channel at its own arrival time adds up at the top channel's arrival."""
import math

import numpy as np

import oracle
from oracle import channels
from paper_1109_3186_gb300 import skymodel

K_DM = skymodel.K_DM


def test_zero_dm_is_a_plain_sum_over_valid_dumps():
    rng = np.random.default_rng(1)
    P = [rng.random((1, 20, 3)) for _ in range(3)]
    first = [np.array([2]), np.array([0]), np.array([4])]
    last = [np.array([19]), np.array([17]), np.array([19])]
    E = channels.combine(P, first, last, [1.3e9, 1.4e9, 1.5e9], 32e6, 1024, K_DM, [0.0])
    want = sum(P)
    assert np.allclose(E[0, 4:18], want[0, 4:18], rtol=0, atol=1e-12)
    assert np.all(E[0, :4] == 0) and np.all(E[0, 18:] == 0)


def test_shifts_follow_the_dispersion_delay_between_channel_centres():
    f_c = channels.channel_centres(1.4e9, 42e6, 8)
    bw, L, dms = 42e6, 4096, [0.0, 100.0, 1000.0, 2000.0]
    s = channels.shifts(f_c, bw, L, K_DM, dms)
    f_ref = f_c.max()
    assert np.all(s[0] == 0) and np.all(s[:, -1] == 0)
    for d, dm in enumerate(dms[1:], start=1):
        assert np.all(np.diff(s[d]) <= 0)            # lower channels arrive later
        for c, f in enumerate(f_c[:-1]):
            # the C oracle's sweep below a band centre f_ref over bandwidth 2 (f_ref - f)
            b2 = 2.0 * (f_ref - f)
            hi, lo = oracle.sweep(f_ref, b2, K_DM, dm)
            assert s[d, c] == int(np.rint(lo / b2 * bw / L))


def _burst_case():
    n_ant, n_samp, bw, L = 4, 1 << 15, 8e6, 1024
    f_c = channels.channel_centres(1.4e9, bw, 3)
    dms = np.array([0.0, 10.0])
    xyz = skymodel.antenna_positions(n_ant, 1500.0, 7)
    pix = skymodel.pixel_grid(3, 0.6)
    true_pix = 4
    t_ref = 12.5 * L                                   # arrival at the top channel's centre, samples
    P, first, last = [], [], []
    for c, f in enumerate(f_c):
        x = skymodel.noise(n_ant, n_samp, 40 + c)
        delay = K_DM * dms[1] * (f ** -2 - f_c.max() ** -2) * bw
        p = skymodel.Pulse(dm=float(dms[1]), t0=t_ref + delay, fwhm_s=40e-6,
                           amp=skymodel.burst_amplitude(25.0, n_ant, L, 40e-6 * bw, L / 2),
                           l=pix[true_pix][0], m=pix[true_pix][1], seed=50 + c)
        skymodel.inject(x, xyz, f, bw, p)
        P.append(oracle.chimageator(x, f, bw, K_DM, dms, 1 << 13, L, xyz, pix))
        lay = [oracle.layout(dms, d, f, bw, K_DM, n_samp, 1 << 13) for d in range(2)]
        fl = [oracle.dump_range(n_samp, lay[d]["n_hi"], lay[d]["n_lo"], L) for d in range(2)]
        first.append(np.array([v[0] for v in fl]))
        last.append(np.array([v[1] for v in fl]))
    E = channels.combine(P, first, last, f_c, bw, L, K_DM, dms)
    return E, P, f_c, bw, L, dms, int(t_ref // L), true_pix


def test_a_burst_across_channels_adds_up_at_the_top_channels_arrival():
    E, P, f_c, bw, L, dms, m, true_pix = _burst_case()
    assert int(np.argmax(E[1, :, true_pix])) == m
    assert int(np.argmax(E[1, m])) == true_pix
    s = channels.shifts(f_c, bw, L, K_DM, dms)
    assert math.isclose(E[1, m, true_pix], sum(P[c][1, m + s[1, c], true_pix] for c in range(3)),
                        rel_tol=1e-12)
    # the aligned sum collects (nearly) every channel's own peak
    peaks = sum(float(P[c][1, :, true_pix].max()) for c in range(3))
    assert E[1, m, true_pix] >= 0.9 * peaks


def test_planted_wrong_sign_shifts_miss_the_burst(monkeypatch):
    good = channels.shifts
    monkeypatch.setattr(channels, "shifts", lambda *a: -good(*a))
    E, P, f_c, bw, L, dms, m, true_pix = _burst_case()
    peaks = sum(float(P[c][1, :, true_pix].max()) for c in range(3))
    assert E[1, :, true_pix].max() < 0.9 * peaks
