"""The coarse-channel combination on the GPU (chirp_combine_channels) against
the FP64 oracle (oracle/channels.py, Eq. dmdelay between channel centres).

Four 4 MHz channels around 1.4 GHz carry one burst, injected into each
channel at that channel's own arrival time.  Each channel is searched by its
own Chimageator plan on its own stream, all four in one chirp_batch_run; the
GPU then aligns the channels' dump powers to the top channel and adds them.
Checked:
- the GPU combination of the GPU powers equals the oracle's combination of
  the same powers (FP32 sums of 4 terms: 1e-6 relative);
- the GPU combination equals the oracle's combination of the oracle's own
  per-channel searches within the FP32 path's 1e-5;
- zeros exactly where the oracle has no combined dump, and the burst adds up
  at the top channel's arrival dump and pixel.
"""
import numpy as np
import pytest

import oracle
import paper_1109_3186_gb300 as chirp
from oracle import channels
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_POW, pow_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K_DM = skymodel.K_DM


def _case():
    n_ant, n_samp, bw, L, nfft_min = 6, 1 << 17, 4e6, 1024, 1 << 14
    f_c = channels.channel_centres(1.4e9, bw, 4)
    dms = np.linspace(0.0, 120.0, 6)
    xyz = skymodel.antenna_positions(n_ant, 2000.0, 21)
    pix = skymodel.pixel_grid(4, 0.8)
    true_pix, dm_true = 6, float(dms[3])
    t_ref = 70.5 * L
    xs = []
    for c, f in enumerate(f_c):
        x = skymodel.noise(n_ant, n_samp, 300 + c)
        delay = K_DM * dm_true * (f ** -2 - f_c.max() ** -2) * bw
        p = skymodel.Pulse(dm=dm_true, t0=t_ref + delay, fwhm_s=60e-6,
                           amp=skymodel.burst_amplitude(30.0, n_ant, L, 60e-6 * bw, L / 2),
                           l=pix[true_pix][0], m=pix[true_pix][1], seed=400 + c)
        skymodel.inject(x, xyz, f, bw, p)
        xs.append(x)
    return dict(n_ant=n_ant, n_samp=n_samp, bw=bw, L=L, nfft_min=nfft_min, f_c=f_c, dms=dms,
                xyz=xyz, pix=pix, true_pix=true_pix, m_ref=int(t_ref // L), xs=xs)


def test_channels_combined_on_the_gpu_match_the_oracle():
    k = _case()
    C = len(k["f_c"])
    plans, outs, volts = [], [], []
    for c in range(C):
        st = torch.cuda.Stream()
        pl = chirp.Plan(k["xyz"], k["f_c"][c], k["bw"], k["n_samp"], k["dms"], k["L"],
                        k["nfft_min"], pix_lm=k["pix"], stream=st)
        plans.append(pl)
        volts.append(torch.from_numpy(k["xs"][c]).cuda())
        outs.append(torch.empty((len(k["dms"]), pl.n_dump, pl.n_pix), dtype=torch.float32,
                                device="cuda"))
    torch.cuda.synchronize()
    chirp.chirp_batch_run(plans, volts, outs, [1] * C)
    torch.cuda.synchronize()
    ranges = [pl.dump_range() for pl in plans]
    first = np.array([r[0] for r in ranges])
    last = np.array([r[1] for r in ranges])
    E = torch.full_like(outs[0], -1.0)
    chirp.chirp_combine_channels(outs, first, last, k["f_c"], k["bw"], k["L"], k["dms"], E,
                                 k_dm=K_DM)
    torch.cuda.synchronize()
    Eg = E.cpu().numpy()
    Pg = [o.cpu().numpy() for o in outs]
    for pl in plans:
        pl.close()

    # the kernel alone: oracle combination of the GPU's own powers
    Ek = channels.combine(Pg, list(first), list(last), k["f_c"], k["bw"], k["L"], K_DM, k["dms"])
    assert np.array_equal(Eg == 0, Ek == 0)
    nz = Ek > 0
    assert np.abs(Eg[nz] - Ek[nz]).max() <= 1e-6 * np.abs(Ek[nz]).max()
    assert (np.abs(Eg[nz] - Ek[nz]) / Ek[nz]).max() <= 1e-6

    # the whole path: oracle searches of every channel, combined by the oracle
    Po = [oracle.chimageator(k["xs"][c], k["f_c"][c], k["bw"], K_DM, k["dms"], k["nfft_min"],
                             k["L"], k["xyz"], k["pix"]) for c in range(C)]
    Eo = channels.combine(Po, list(first), list(last), k["f_c"], k["bw"], k["L"], K_DM, k["dms"])
    assert np.array_equal(Eg == 0, Eo == 0)
    assert pow_error(Eg, Eo) <= TOL_POW

    # the burst: at its DM and pixel the combined power peaks at the top channel's arrival
    d = 3
    assert int(np.argmax(Eo[d, :, k["true_pix"]])) == k["m_ref"]
    assert int(np.argmax(Eg[d, :, k["true_pix"]])) == k["m_ref"]
    s = channels.shifts(k["f_c"], k["bw"], k["L"], K_DM, k["dms"])
    assert s[d, 0] > 0  # the lowest channel arrives dumps later


def test_combine_refuses_bad_arguments():
    P = [torch.zeros((2, 8, 4), dtype=torch.float32, device="cuda") for _ in range(2)]
    E = torch.zeros_like(P[0])
    first = np.zeros((2, 2), np.int64)
    last = np.full((2, 2), 7, np.int64)
    with pytest.raises(chirp.ChirpError):
        chirp.chirp_combine_channels(P, first - 1, last, [1.4e9, 1.41e9], 1e7, 64, [0.0, 1.0], E)
    with pytest.raises(chirp.ChirpError):
        chirp.chirp_combine_channels(P, first, last, [1.4e9, -1.0], 1e7, 64, [0.0, 1.0], E)
