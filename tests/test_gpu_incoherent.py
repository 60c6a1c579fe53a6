"""GPU parity of the antenna-incoherent search (power-beam filterbank and
shift-and-sum dedispersion, Sec. 2.3.1 / Sec. 2.4.1) against the FP64 oracle,
through the C ABI, with host and device outputs."""
import numpy as np
import pytest

import oracle as orc
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5   # FP32 sums of n_ant * n_int squared DFT magnitudes


@pytest.mark.parametrize("n_chan,n_int,M,N", [(32, 16, 12, 1 << 17), (16, 4, 3, 50000),
                                              (64, 8, 6, 1 << 16), (256, 2, 2, 40000)])
def test_incoherent_matches_oracle(n_chan, n_int, M, N, k_dm):
    sc = skymodel.chimageator_medium(n_samp=N, n_dm=2, n_ant=M, dm_max=60.0, nfft_min=1 << 14,
                                     dump_len=1024, n_side=2, n_pulse=1)
    for p in sc.pulses:
        p.amp *= 4
    x = sc.voltages()
    fb_dms = np.linspace(0.0, 300.0, 17)
    plan = chirp.Plan.from_scenario(sc, fb_chan=n_chan, fb_int=n_int, fb_dm=fb_dms)
    T = plan.info["fb_samples"]
    assert T == N // (n_chan * n_int)
    S_o = orc.filterbank(x, n_chan, n_int)
    D_o = orc.incoherent(S_o, sc.f0, sc.bw, k_dm, n_int, fb_dms)
    # device buffers
    Sd = torch.empty((n_chan, T), dtype=torch.float32, device="cuda")
    Dd = torch.empty((fb_dms.size, T), dtype=torch.float32, device="cuda")
    plan.incoherent(torch.from_numpy(x).cuda(), Dd, Sd)
    S_g, D_g = Sd.cpu().numpy(), Dd.cpu().numpy()
    assert np.abs(S_g - S_o).max() <= TOL * S_o.max()
    assert np.all((D_o == 0) == (D_g == 0))
    m = D_o > 0
    assert (np.abs(D_g - D_o)[m] / D_o[m]).max() < TOL
    # host buffers, same numbers
    Dh = np.empty((fb_dms.size, T), np.float32)
    plan.incoherent(x, Dh)
    assert np.array_equal(Dh, D_g)


def test_incoherent_finds_the_burst(k_dm):
    """The injected burst peaks at its own DM near its arrival time."""
    sc = skymodel.chimageator_medium(n_samp=1 << 19, n_dm=2, n_ant=12, dm_max=200.0,
                                     nfft_min=1 << 16, dump_len=4096, n_side=2, n_pulse=1,
                                     seed=77)
    p = sc.pulses[0]
    p.amp *= 3
    x = sc.voltages()
    fb_dms = np.linspace(0.0, 300.0, 61)
    plan = chirp.Plan.from_scenario(sc, fb_chan=32, fb_int=16, fb_dm=fb_dms)
    T = plan.info["fb_samples"]
    D = np.empty((fb_dms.size, T), np.float32)
    plan.incoherent(x, D)
    z = (D - np.median(D[D > 0])) / D[D > 0].std()
    z[D == 0] = 0
    d, t = np.unravel_index(np.argmax(z), z.shape)
    assert abs(fb_dms[d] - p.dm) <= 2 * (fb_dms[1] - fb_dms[0])
    assert abs(t * 32 * 16 - p.t0) <= 2 * 32 * 16
