"""GPU parity of the two back-ends, through the C ABI, against the FP64
oracle: Chirpolator visibilities (Eq. xpq products integrated per dump) and
Chimageator beam powers (Sec. 2.4.2 phased sum, |.|^2, integrated).  FP32
path tolerance 1e-5 on both metrics."""
import numpy as np
import pytest

import oracle as orc
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_POW, TOL_VIS, pow_error, vis_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


CORR_CASES = [
    (6, 1 << 17, 1024, [0.0, 20.0, 40.0, 75.0], 1 << 14),
    (4, 100003, 777, [0.0, 33.0], 1 << 13),     # ragged N and dump length
    (8, 50000, 1000, [0.0, 12.0], 1 << 13),     # even dump length, not a multiple of 256
    (1, 1 << 15, 512, [5.0], 1 << 12),          # one antenna: autos only
    (13, 1 << 15, 256, [0.0, 9.0], 1 << 12),    # 91 pairs
    (36, 1 << 14, 1024, [0.0, 5.0], 1 << 12),   # 666 pairs; tensor cores: two row tiles
    (48, 1 << 14, 2048, [0.0, 3.0], 1 << 12),   # largest split-BF16 tensor-core shape
]


@pytest.mark.parametrize("corr", [chirp.CORR_FP32_SIMT, chirp.CORR_TC_3XBF16],
                         ids=["fp32_simt", "tc_3xbf16"])
@pytest.mark.parametrize("M,N,L,dms,nfft_min", CORR_CASES,
                         ids=["M%d_N%d_L%d" % (c[0], c[1], c[2]) for c in CORR_CASES])
def test_chirpolator_matches_oracle(M, N, L, dms, nfft_min, corr, k_dm):
    if corr == chirp.CORR_TC_3XBF16 and L % 128 and 256 % L:
        pytest.skip("tensor-core correlation needs dump chunks that line up")
    sc = skymodel.chirpolator_small(n_samp=N, n_dm=len(dms), n_ant=M, dm_max=max(dms),
                                    nfft_min=nfft_min, dump_len=L)
    sc.dms = np.array(dms)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, corr_mode=corr)
    assert plan.info["corr_mode"] == corr
    V = torch.empty((len(dms), plan.n_dump, plan.n_pair), dtype=torch.complex64, device="cuda")
    plan.chirpolator(torch.from_numpy(x).cuda(), V)
    Vg = V.cpu().numpy()
    Vo = orc.chirpolator(x, sc.f0, sc.bw, k_dm, sc.dms, nfft_min, L)
    first, last = plan.dump_range()
    for d in range(len(dms)):
        assert np.all(Vg[d, :first[d]] == 0) and np.all(Vg[d, last[d] + 1:] == 0)
    assert vis_error(Vg, Vo, M) < TOL_VIS


BEAM_CASES = [
    (12, 1 << 17, 4096, 8, [0.0, 30.0, 60.0], 1 << 15),
    (5, 50000, 1000, 3, [0.0, 12.0], 1 << 13),        # 9 pixels: one padded row tile
    (3, 1 << 14, 512, 1, [7.0], 1 << 12),
    (13, 70000, 777, 12, [0.0, 20.0], 1 << 14),       # dumps straddle 128-sample tiles
    (12, 1 << 18, 4096, 32, [0.0, 150.0, 300.0], 1 << 17),   # 1024 beams, all row tiles
    (7, 1 << 16, 2048, 20, [0.0, 25.0], 1 << 14),     # 400 beams: 7 row tiles (odd)
    (12, 1 << 17, 512, 40, [40.0], 1 << 15),          # 1600 beams: 25 row tiles, 4 CTAs wide
]


# (beam mode, tensor-core kernel shape): 0 = the library's choice, 1 = 128-sample
# tiles with the weights in shared memory, 2 = 256-sample tiles, 3 = 128-sample
# tiles with the weights in TMEM
MODES = [(chirp.BEAM_FP32_SIMT, 0), (chirp.BEAM_TC_3XBF16, 0), (chirp.BEAM_TC_3XBF16, 1),
         (chirp.BEAM_TC_3XBF16, 2), (chirp.BEAM_TC_3XBF16, 3), (chirp.BEAM_VIS, 0)]


@pytest.mark.parametrize("mode,shape", MODES,
                         ids=["fp32_simt", "tc_3xbf16", "tc_smem128", "tc_smem256", "tc_tmem128",
                              "vis"])
@pytest.mark.parametrize("M,N,L,n_side,dms,nfft_min", BEAM_CASES,
                         ids=["M%d_N%d_L%d_pix%d" % (c[0], c[1], c[2], c[3] ** 2) for c in BEAM_CASES])
def test_chimageator_matches_oracle(M, N, L, n_side, dms, nfft_min, mode, shape, k_dm):
    if shape == 2 and L % 256:
        pytest.skip("256-sample tiles need dump_len % 256 == 0")
    sc = skymodel.chimageator_medium(n_samp=N, n_dm=len(dms), n_ant=M, dm_max=max(dms),
                                     nfft_min=nfft_min, dump_len=L, n_side=n_side, n_pulse=1)
    sc.dms = np.array(dms)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, beam_mode=mode, beam_shape=shape)
    assert plan.info["beam_mode"] == mode
    if mode == chirp.BEAM_TC_3XBF16:
        assert plan.info["beam_shape"] == (shape or (2 if L % 256 == 0 else 1))
    P = torch.empty((len(dms), plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    plan.chimageator(torch.from_numpy(x).cuda(), P)
    Pg = P.cpu().numpy()
    Po = orc.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, nfft_min, L, sc.xyz, sc.pix_lm)
    plan.status()
    first, last = plan.dump_range()
    for d in range(len(dms)):
        assert np.all(Pg[d, :first[d]] == 0) and np.all(Pg[d, last[d] + 1:] == 0)
        assert np.all(Pg[d, first[d]:last[d] + 1] > 0)
    assert pow_error(Pg, Po) < TOL_POW


def test_host_buffers_round_trip(k_dm):
    """Host input and host output through the same entry points."""
    sc = skymodel.chirpolator_small(n_samp=1 << 15, n_dm=2, n_ant=3, dm_max=20.0,
                                    nfft_min=1 << 13, dump_len=512)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc)
    Vh = np.empty((2, plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, Vh)
    Vd = torch.empty(Vh.shape, dtype=torch.complex64, device="cuda")
    plan.chirpolator(torch.from_numpy(x).cuda(), Vd)
    assert np.array_equal(Vh, Vd.cpu().numpy())


def test_auto_correlation_mode_and_refusals():
    sc = skymodel.chirpolator_small(n_samp=1 << 15, n_dm=2, n_ant=12, dm_max=10.0,
                                    nfft_min=1 << 12, dump_len=777)
    assert chirp.Plan.from_scenario(sc).info["corr_mode"] == chirp.CORR_FP32_SIMT
    with pytest.raises(chirp.ChirpError) as ei:
        chirp.Plan.from_scenario(sc, corr_mode=chirp.CORR_TC_3XBF16)
    assert ei.value.code == -5
    sc.dump_len = 1024
    # up to 16 antennas AUTO keeps the (faster) staged FP32 correlator
    assert chirp.Plan.from_scenario(sc).info["corr_mode"] == chirp.CORR_FP32_SIMT
    assert chirp.Plan.from_scenario(sc, corr_mode=chirp.CORR_TC_3XBF16).info["corr_mode"] == \
        chirp.CORR_TC_3XBF16
    sc20 = skymodel.chirpolator_small(n_samp=1 << 15, n_dm=2, n_ant=20, dm_max=10.0,
                                      nfft_min=1 << 12, dump_len=1024)
    assert chirp.Plan.from_scenario(sc20).info["corr_mode"] == chirp.CORR_TC_3XBF16


_LONG = {}


def _long_case(M, N, dms, nfft_min, n_side, k_dm):
    """Scenario, voltages and oracle powers of a case whose FFT groups have
    column lengths of 1024 or more (the column pass writes the beam image
    sample by sample there), computed once per module."""
    key = (M, N, tuple(dms), nfft_min, n_side)
    if key not in _LONG:
        sc = skymodel.chimageator_medium(n_samp=N, n_dm=len(dms), n_ant=M, dm_max=max(dms),
                                         nfft_min=nfft_min, dump_len=4096, n_side=n_side,
                                         n_pulse=1)
        sc.dms = np.array(dms)
        x = sc.voltages()
        Po = orc.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, nfft_min, 4096, sc.xyz, sc.pix_lm)
        _LONG[key] = (sc, x, Po)
    return _LONG[key]


LONG_CASES = [
    (4, 1 << 23, [0.0, 300.0, 700.0], 1 << 22, 2),   # columns of 1024 (3 blocks) and 2048
    (2, 1 << 24, [0.0, 900.0], 1 << 24, 1),          # columns of 4096: one 2^24 block
]


@pytest.mark.parametrize("mode", [chirp.BEAM_TC_3XBF16, chirp.BEAM_TC_BF16],
                         ids=["tc_3xbf16", "tc_bf16"])
@pytest.mark.parametrize("M,N,dms,nfft_min,n_side", LONG_CASES,
                         ids=["M%d_N%d" % (c[0], c[1]) for c in LONG_CASES])
def test_chimageator_long_transforms(M, N, dms, nfft_min, n_side, mode, k_dm):
    sc, x, Po = _long_case(M, N, dms, nfft_min, n_side, k_dm)
    plan = chirp.Plan.from_scenario(sc, beam_mode=mode)
    assert plan.info["beam_mode"] == mode
    assert max(plan.dm_layout(d)["nfft"] for d in range(len(dms))) >= 1 << 23
    P = torch.empty((len(dms), plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    plan.chimageator(torch.from_numpy(x).cuda(), P)
    plan.status()
    Pg = P.cpu().numpy()
    first, last = plan.dump_range()
    for d in range(len(dms)):
        assert np.all(Pg[d, :first[d]] == 0) and np.all(Pg[d, last[d] + 1:] == 0)
    tol = TOL_POW if mode == chirp.BEAM_TC_3XBF16 else 1e-2
    assert pow_error(Pg, Po) < tol
    plan.close()
