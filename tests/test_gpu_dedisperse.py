"""GPU parity of the coherent-dedispersion stage (overlap-save FFT, chirp
multiply, IFFT; Sec. 2.3.2 with Eq. 1) against the FP64 oracle, called
through the C ABI.  Sizes span every FFT tile (column and row lengths
16..4096), multi-block grids with ragged last blocks, single zero-padded
blocks, DM = 0 and DMs with no valid output."""
import numpy as np
import pytest

import oracle as orc
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_Y_MAX, TOL_Y_RMS, y_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _noise(M, N, seed):
    return skymodel.noise(M, N, seed)


CASES = [
    # f0, bw, M, N, dms, nfft_min
    (1.4e9, 8e6, 2, 3000, [0.0, 1.0, 2.5], 256),           # tiny, 16 x 16 split
    (1.4e9, 8e6, 3, 20000, [0.0, 3.0, 9.0], 1024),         # 16 x 64
    (1.4e9, 8e6, 2, 50000, [5.0, 12.0], 4096),             # 16 x 256
    (1.4e9, 8e6, 2, 70001, [0.0, 20.0, 30.0], 1 << 14),    # 16 x 1024, ragged N
    (1.4e9, 8e6, 2, 1 << 17, [0.0, 40.0, 75.0], 1 << 16),  # 16 x 4096
    (1.4e9, 32e6, 2, 1 << 19, [0.0, 10.0, 30.0], 1 << 17), # 32 x 4096
    (1.4e9, 32e6, 1, 1 << 20, [0.0, 60.0], 1 << 18),       # 64 x 4096 and 2^19
    (1.4e9, 32e6, 1, 1 << 20, [150.0], 1 << 18),           # 2^20 = 256 x 4096 single block
    (1.4e9, 32e6, 1, 1 << 23, [0.0, 300.0, 700.0], 1 << 22),  # 1024 x 4096 (3 blocks), 2048 x 4096
    (1.4e9, 32e6, 1, 1 << 24, [0.0, 900.0], 1 << 24),      # 4096 x 4096: the largest transform
]


@pytest.mark.parametrize("case", CASES, ids=[f"N{c[3]}_nfft{c[5]}" for c in CASES])
def test_dedispersion_matches_oracle(case, k_dm):
    f0, bw, M, N, dms, nfft_min = case
    x = _noise(M, N, 17 + N % 1000)
    plan = chirp.Plan(np.zeros((M, 3)), f0, bw, N, dms, 256, nfft_min)
    xd = torch.from_numpy(x).cuda()
    for d in range(len(dms)):
        lay_o = orc.layout(dms, d, f0, bw, k_dm, N, nfft_min)
        assert plan.dm_layout(d) == lay_o
        y = torch.empty((M, N), dtype=torch.complex64, device="cuda")
        plan.dedisperse(xd, d, y)
        torch.cuda.synchronize()
        yg = y.cpu().numpy()
        yo = orc.dedisperse(x, f0, bw, k_dm, dms, d, nfft_min)
        inval = yo == 0
        assert np.all(yg[inval] == 0)
        rms, mx = y_error(yg, yo)
        assert rms < TOL_Y_RMS and mx < TOL_Y_MAX, (d, rms, mx)


def test_dm_without_valid_output(k_dm):
    N = 40000
    x = _noise(2, N, 3)
    dms = [0.0, 500.0]             # sweep at 500 exceeds the whole series
    plan = chirp.Plan(np.zeros((2, 3)), 1.4e9, 8e6, N, dms, 1000, 1 << 12)
    first, last = plan.dump_range()
    assert last[1] < first[1]
    y = np.empty((2, N), np.complex64)
    plan.dedisperse(x, 1, y)       # host in, host out
    assert np.all(y == 0)
    plan.dedisperse(x, 0, y)
    assert np.abs(y - x).max() < 1e-6


def test_dispersed_pulse_is_recovered(k_dm):
    """A sky-model burst dedispersed at its true DM peaks at its arrival time."""
    sc = skymodel.chirpolator_small(n_samp=1 << 18, n_dm=5, dm_max=60.0, nfft_min=1 << 15)
    p = sc.pulses[0]
    p.amp *= 10
    x = sc.voltages()
    d = int(np.argmin(np.abs(sc.dms - p.dm)))
    plan = chirp.Plan.from_scenario(sc)
    y = np.empty_like(x)
    plan.dedisperse(x, d, y)
    e = (np.abs(y) ** 2).sum(0)
    assert abs(int(np.argmax(e)) - p.t0) < 3 * p.fwhm_s * sc.bw
