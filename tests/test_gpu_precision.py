"""The precision form: complex int8 voltage ingest and BF16 beam contraction.

- int8 input (value = scale[a] * (re + j im)) is converted to FP32 inside the
  first FFT pass; every output equals, bit for bit, the same plan's output on
  the complex64 voltages that conversion produces, and matches the oracle run
  on those voltages.
- The one-term BF16 tensor-core beamformer (operands rounded once to BF16,
  FP32 accumulation) matches the oracle's beam powers to 1e-2 relative: a
  BF16 operand carries a relative rounding error of at most 2^-9 = 2e-3, a
  beam voltage sums M such products with independent errors, and a power
  doubles the voltage's relative error, so single samples err by a few 1e-3
  and dump sums (thousands of samples) by less.
"""
import numpy as np
import pytest

import oracle as orc
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_POW, TOL_VIS, pow_error, vis_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_POW_BF16 = 1e-2
TOL_VIS_BF16 = 1e-2


def _int8(sc):
    q, s = skymodel.quantize_ci8(sc.voltages())
    return q, s, skymodel.dequantize_ci8(q, s)


@pytest.mark.parametrize("loc", ["device", "host"])
def test_int8_chirpolator_equals_dequantised_and_oracle(loc, k_dm):
    sc = skymodel.chirpolator_small(n_samp=100003, n_dm=4, dm_max=75.0, nfft_min=1 << 14,
                                    dump_len=777)
    q, s, xf = _int8(sc)
    p8 = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=s)
    pf = chirp.Plan.from_scenario(sc)
    V8 = np.empty((len(sc.dms), p8.n_dump, p8.n_pair), np.complex64)
    Vf = np.empty_like(V8)
    p8.chirpolator(torch.from_numpy(q).cuda() if loc == "device" else q, V8)
    pf.chirpolator(xf, Vf)
    assert np.array_equal(V8, Vf)
    Vo = orc.chirpolator(xf.astype(np.complex128), sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min,
                         sc.dump_len)
    assert vis_error(V8, Vo, sc.n_ant) < TOL_VIS


def test_int8_dedispersion_and_incoherent_equal_dequantised():
    sc = skymodel.chirpolator_small(n_samp=1 << 17, n_dm=3, dm_max=60.0, nfft_min=1 << 14)
    q, s, xf = _int8(sc)
    kw = dict(fb_chan=32, fb_int=8, fb_dm=sc.dms)
    p8 = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=s, **kw)
    pf = chirp.Plan.from_scenario(sc, **kw)
    qd, xd = torch.from_numpy(q).cuda(), torch.from_numpy(xf).cuda()
    y8 = torch.empty((sc.n_ant, sc.n_samp), dtype=torch.complex64, device="cuda")
    yf = torch.empty_like(y8)
    p8.dedisperse(qd, 2, y8)
    pf.dedisperse(xd, 2, yf)
    assert torch.equal(y8, yf)
    T = p8.info["fb_samples"]
    D8 = torch.empty((len(sc.dms), T), dtype=torch.float32, device="cuda")
    Df = torch.empty_like(D8)
    p8.incoherent(qd, D8)
    pf.incoherent(xd, Df)
    assert torch.equal(D8, Df)


def test_int8_plan_rejects_complex64_input():
    sc = skymodel.chirpolator_small(n_samp=1 << 15, n_dm=2, dm_max=10.0, nfft_min=1 << 12)
    p8 = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8)
    V = np.empty((2, p8.n_dump, p8.n_pair), np.complex64)
    with pytest.raises(TypeError):
        p8.chirpolator(sc.voltages(), V)


BF16_CASES = [
    (12, 1 << 17, 4096, 8, [0.0, 30.0, 60.0], 1 << 15),   # G = 3: zero padding k-group
    (8, 50000, 1000, 3, [0.0, 12.0], 1 << 13),            # G = 2, 128-sample tiles
    (5, 1 << 16, 512, 20, [0.0, 25.0], 1 << 14),          # 400 beams, 7 row tiles
    (36, 1 << 16, 1024, 8, [0.0, 3.0], 1 << 14),          # G = 9
]


@pytest.mark.parametrize("M,N,L,n_side,dms,nfft_min", BF16_CASES,
                         ids=["M%d_L%d_pix%d" % (c[0], c[2], c[3] ** 2) for c in BF16_CASES])
def test_bf16_beams_match_oracle(M, N, L, n_side, dms, nfft_min, k_dm):
    sc = skymodel.chimageator_medium(n_samp=N, n_dm=len(dms), n_ant=M, dm_max=max(dms),
                                     nfft_min=nfft_min, dump_len=L, n_side=n_side, n_pulse=1)
    sc.dms = np.array(dms)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, beam_mode=chirp.BEAM_TC_BF16)
    assert plan.info["beam_mode"] == chirp.BEAM_TC_BF16
    P = torch.empty((len(dms), plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    plan.chimageator(torch.from_numpy(x).cuda(), P)
    plan.status()
    Pg = P.cpu().numpy()
    Po = orc.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, nfft_min, L, sc.xyz, sc.pix_lm)
    first, last = plan.dump_range()
    for d in range(len(dms)):
        assert np.all(Pg[d, :first[d]] == 0) and np.all(Pg[d, last[d] + 1:] == 0)
    err = pow_error(Pg, Po)
    assert err < TOL_POW_BF16, err


@pytest.mark.parametrize("M,L", [(12, 1024), (36, 2048), (84, 512)])
def test_bf16_correlation_matches_oracle(M, L, k_dm):
    sc = skymodel.chirpolator_small(n_samp=1 << 15, n_dm=2, n_ant=M, dm_max=10.0,
                                    nfft_min=1 << 12, dump_len=L)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, corr_mode=chirp.CORR_TC_BF16)
    V = np.empty((2, plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, V)
    plan.status()
    Vo = orc.chirpolator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len)
    err = vis_error(V, Vo, M)
    assert err < TOL_VIS_BF16, err


def test_precision_form_channel(k_dm):
    """One coarse channel of the 36-antenna int8 array (reduced length and DM
    range): int8 ingest, FP32 Chirpolator, BF16 Chimageator."""
    sc = skymodel.precision_form(channel=5, n_samp=1 << 17, n_dm=6, dm_min=0.5, dm_max=6.0,
                                 n_side=8, dump_len=2048, nfft_min=1 << 14)
    q, s, xf = _int8(sc)
    xo = xf.astype(np.complex128)
    qd = torch.from_numpy(q).cuda()
    pv = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=s)
    V = torch.empty((len(sc.dms), pv.n_dump, pv.n_pair), dtype=torch.complex64, device="cuda")
    pv.chirpolator(qd, V)
    Vo = orc.chirpolator(xo, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len)
    assert vis_error(V.cpu().numpy(), Vo, sc.n_ant) < TOL_VIS
    # the precision form's correlation: BF16 on the tensor cores
    pb16 = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=s,
                                    corr_mode=chirp.CORR_TC_BF16)
    V16 = torch.empty_like(V)
    pb16.chirpolator(qd, V16)
    pb16.status()
    assert vis_error(V16.cpu().numpy(), Vo, sc.n_ant) < TOL_VIS_BF16
    pb = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=s,
                                  beam_mode=chirp.BEAM_TC_BF16)
    P = torch.empty((len(sc.dms), pb.n_dump, pb.n_pix), dtype=torch.float32, device="cuda")
    pb.chimageator(qd, P)
    pb.status()
    Po = orc.chimageator(xo, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len, sc.xyz,
                         sc.pix_lm)
    assert pow_error(P.cpu().numpy(), Po) < TOL_POW_BF16
    # the split-BF16 mode on the same int8 input stays at the FP32 tolerance
    p3 = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=s,
                                  beam_mode=chirp.BEAM_TC_3XBF16)
    P3 = torch.empty_like(P)
    p3.chimageator(qd, P3)
    assert pow_error(P3.cpu().numpy(), Po) < TOL_POW


def test_precision_form_slice_of_the_36_antenna_array(k_dm):
    """The measurement slice of the 36-antenna precision form: one coarse
    channel, 2^20 int8 samples, 8 trial DMs spanning its 0-2000 grid (FFT
    groups 2^16 ... 2^20; the last group is one block holding four DMs, three
    of which have no valid dump), 64 x 64 beams.  Sampled dumps of every DM
    with valid output (its first, middle and last dumps, and the burst's dump)
    against the oracle on the dequantised voltages: BF16 beams and BF16
    correlation within 1e-2, split-BF16 beams and correlation within 1e-5;
    DMs without valid dumps are all zero."""
    sc = skymodel.precision_form(channel=3, n_samp=1 << 20, n_dm=256)
    sc.dms = sc.dms[np.unique(np.linspace(0, 255, 8).round().astype(int))]
    q, s, xf = _int8(sc)
    qd = torch.from_numpy(q).cuda()
    n_dm = len(sc.dms)
    out = {}
    for name, kw in (("p16", dict(beam_mode=chirp.BEAM_TC_BF16)),
                     ("p3", dict(beam_mode=chirp.BEAM_TC_3XBF16)),
                     ("v16", dict(corr_mode=chirp.CORR_TC_BF16)),
                     ("v3", dict(corr_mode=chirp.CORR_TC_3XBF16))):
        plan = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=s, **kw)
        if name.startswith("p"):
            o = torch.empty((n_dm, plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
            plan.chimageator(qd, o)
        else:
            o = torch.empty((n_dm, plan.n_dump, plan.n_pair), dtype=torch.complex64, device="cuda")
            plan.chirpolator(qd, o)
        plan.status()
        out[name] = o.cpu().numpy()
        first, last = plan.dump_range()
        plan.close()
    lay = [orc.layout(sc.dms, d, sc.f0, sc.bw, k_dm, sc.n_samp, sc.nfft_min) for d in range(n_dm)]
    assert len({l["nfft"] for l in lay}) == 4 and lay[-1]["n_blk"] == 1
    valid = [d for d in range(n_dm) if last[d] >= first[d]]
    assert len(valid) == 5 and valid == list(range(5))
    for d in range(5, n_dm):
        for o in out.values():
            assert np.all(o[d] == 0)
    L = sc.dump_len
    W = orc.beam_weights(sc.xyz, sc.pix_lm, sc.f0)
    x128 = xf.astype(np.complex128)
    p = sc.pulses[0]
    d_p = int(np.argmin(np.abs(sc.dms - p.dm)))
    for d in valid:
        y = orc.dedisperse(x128, sc.f0, sc.bw, k_dm, sc.dms, d, sc.nfft_min)
        f, l = int(first[d]), int(last[d])
        spans = [(f, f + 1), ((f + l) // 2, (f + l) // 2 + 1), (l, l + 1)]
        if d == d_p:
            spans.append((int(p.t0 // L), int(p.t0 // L) + 1))
        for m0, m1 in spans:
            ys = y[:, m0 * L:m1 * L]
            Po = orc.beamform(ys, W, L, m0, m1, f, l)
            Vo = orc.correlate(ys, L, m0, m1, f, l)
            assert pow_error(out["p16"][d, m0:m1], Po) < TOL_POW_BF16, (d, m0)
            assert pow_error(out["p3"][d, m0:m1], Po) < TOL_POW, (d, m0)
            assert vis_error(out["v16"][d, m0:m1], Vo, sc.n_ant) < TOL_VIS_BF16, (d, m0)
            assert vis_error(out["v3"][d, m0:m1], Vo, sc.n_ant) < TOL_VIS, (d, m0)


VIS_BF16_CASES = [
    (12, 1 << 17, 4096, 8, [0.0, 30.0, 60.0], 1 << 15),   # staged correlator, 16-byte copies
    (5, 50001, 1000, 4, [0.0, 12.0], 1 << 13),            # odd series: 4-byte copies
    (36, 1 << 16, 1024, 8, [0.0, 3.0], 1 << 14),          # above 16 antennas: direct loads
]


@pytest.mark.parametrize("M,N,L,n_side,dms,nfft_min", VIS_BF16_CASES,
                         ids=["M%d_N%d" % (c[0], c[1]) for c in VIS_BF16_CASES])
def test_bf16_voltage_visibility_beams_match_oracle(M, N, L, n_side, dms, nfft_min, k_dm):
    """CHIRP_BEAM_VIS_BF16: dedispersed voltages rounded once to BF16 (relative
    error <= 2^-9 per component), FP32 correlation and quadratic form; a dump
    power sums L products whose rounding errors are independent, so its error
    is ~2^-8 / sqrt(L) relative, far inside the reduced-precision 1e-2.  The
    selective search over a seeded mask gives the full search's values."""
    sc = skymodel.chimageator_medium(n_samp=N, n_dm=len(dms), n_ant=M, dm_max=max(dms),
                                     nfft_min=nfft_min, dump_len=L, n_side=n_side, n_pulse=1)
    sc.dms = np.array(dms)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, beam_mode=chirp.BEAM_VIS_BF16)
    assert plan.info["beam_mode"] == chirp.BEAM_VIS_BF16
    xd = torch.from_numpy(x).cuda()
    P = torch.empty((len(dms), plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    plan.chimageator(xd, P)
    Pg = P.cpu().numpy()
    Po = orc.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, nfft_min, L, sc.xyz, sc.pix_lm)
    first, last = plan.dump_range()
    for d in range(len(dms)):
        assert np.all(Pg[d, :first[d]] == 0) and np.all(Pg[d, last[d] + 1:] == 0)
    err = pow_error(Pg, Po)
    assert err < TOL_POW_BF16, err
    assert err > 1e-7  # the voltages really were rounded
    rng = np.random.default_rng(M)
    mask = (rng.random((len(dms), plan.n_dump)) < 0.3).astype(np.uint8)
    S = torch.empty_like(P)
    plan.chimageator_selective(xd, mask, S)
    valid = np.zeros_like(mask, bool)
    for d in range(len(dms)):
        valid[d, first[d]:last[d] + 1] = True
    pick = mask.astype(bool) & valid
    Sg = S.cpu().numpy()
    assert np.all(Sg[~pick] == 0)
    assert np.array_equal(Sg[pick], Pg[pick])
    # the Chirpolator of the same plan keeps FP32 voltages
    V = np.empty((len(dms), plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, V)
    Vo = orc.chirpolator(x, sc.f0, sc.bw, k_dm, sc.dms, nfft_min, L)
    assert vis_error(V, Vo, M) < TOL_VIS
