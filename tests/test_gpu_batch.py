"""Batching, CUDA-graph replay and the FFT-split choice.

- A search replayed as a CUDA graph computes bit for bit what the same plan
  computes with direct launches, and reads the input buffer's current
  contents on every replay.
- chirp_batch_run over observations of uneven shapes, each plan on its own
  stream, computes bit for bit what each search computes alone, and matches
  the oracle.
- Every two-pass split Nfft = n_col * n_row (forced, or chosen by the
  autotuner) matches the oracle to the FP32 tolerance.
"""
import numpy as np
import pytest

import oracle as orc
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_POW, TOL_VIS, pow_error, vis_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _small(M=6, N=1 << 17, n_dm=4, L=1024, nfft_min=1 << 14, seed=1001, **kw):
    return skymodel.chirpolator_small(n_samp=N, n_dm=n_dm, n_ant=M, dm_max=75.0,
                                      nfft_min=nfft_min, dump_len=L, seed=seed, **kw)


def _beams(M=8, N=1 << 17, n_dm=3, L=2048, n_side=8, nfft_min=1 << 15, seed=1002):
    return skymodel.chimageator_medium(n_samp=N, n_dm=n_dm, n_ant=M, dm_max=150.0,
                                       nfft_min=nfft_min, dump_len=L, n_side=n_side, n_pulse=1,
                                       seed=seed)


@pytest.mark.parametrize("backend", ["chirpolator", "chimageator"])
def test_graph_replay_equals_direct_launches(backend):
    sc = _small() if backend == "chirpolator" else _beams()
    st = torch.cuda.Stream()
    direct = chirp.Plan.from_scenario(sc, stream=st, beam_mode=chirp.BEAM_TC_3XBF16)
    graphed = chirp.Plan.from_scenario(sc, stream=st, beam_mode=chirp.BEAM_TC_3XBF16,
                                       flags=chirp.FLAG_GRAPHS)
    if backend == "chirpolator":
        shape, dt = (len(sc.dms), direct.n_dump, direct.n_pair), torch.complex64
    else:
        shape, dt = (len(sc.dms), direct.n_dump, direct.n_pix), torch.float32
    xd = torch.from_numpy(sc.voltages()).cuda()
    ref = torch.empty(shape, dtype=dt, device="cuda")
    out = torch.empty_like(ref)
    torch.cuda.synchronize()
    run_d = getattr(direct, backend)
    run_g = getattr(graphed, backend)
    x_new = torch.from_numpy(_small(seed=77).voltages() if backend == "chirpolator"
                             else _beams(seed=78).voltages()).cuda()
    for it in range(4):  # eager, capture + launch, two replays
        if it == 3:      # new contents in the same input buffer
            xd.copy_(x_new)
        out.zero_()
        torch.cuda.synchronize()
        run_g(xd, out)
        run_d(xd, ref)
        st.synchronize()
        assert torch.equal(out, ref), it
    graphed.status()


def test_graphs_need_a_stream_of_their_own():
    sc = _small(N=1 << 15, nfft_min=1 << 12)
    with pytest.raises(chirp.ChirpError) as ei:
        chirp.Plan.from_scenario(sc, stream=0, flags=chirp.FLAG_GRAPHS)
    assert "stream" in str(ei.value)


# (backend, M, N, bw, n_dm, dm_max, L, nfft_min, n_side)
BATCH = [
    ("chirpolator", 4, 1 << 16, 8e6, 3, 60.0, 512, 1 << 13, 0),
    ("chimageator", 9, 100000, 16e6, 5, 120.0, 1024, 1 << 14, 6),
    ("chirpolator", 11, 1 << 17, 32e6, 2, 20.0, 2048, 1 << 15, 0),
    ("chimageator", 5, 1 << 16, 4e6, 4, 300.0, 4096, 1 << 12, 4),
    ("chirpolator", 2, 70001, 8e6, 6, 150.0, 777, 1 << 13, 0),
]


def _batch_scenario(i, spec):
    be, M, N, bw, n_dm, dm_max, L, nfft_min, n_side = spec
    sc = skymodel.chimageator_medium(n_samp=N, n_dm=n_dm, n_ant=M, dm_max=dm_max,
                                     nfft_min=nfft_min, dump_len=L, n_side=max(n_side, 1),
                                     n_pulse=1, seed=2000 + i, bw=bw)
    return sc


def test_batch_of_uneven_observations(k_dm):
    streams = [torch.cuda.Stream() for _ in BATCH]
    scs = [_batch_scenario(i, spec) for i, spec in enumerate(BATCH)]
    plans, xs, outs, refs, bes = [], [], [], [], []
    for sc, spec, st in zip(scs, BATCH, streams):
        be = 0 if spec[0] == "chirpolator" else 1
        pl = chirp.Plan.from_scenario(sc, stream=st, beam_mode=chirp.BEAM_TC_3XBF16,
                                      flags=chirp.FLAG_GRAPHS)
        shape = (len(sc.dms), pl.n_dump, pl.n_pair if be == 0 else pl.n_pix)
        dt = torch.complex64 if be == 0 else torch.float32
        plans.append(pl)
        bes.append(be)
        xs.append(torch.from_numpy(sc.voltages()).cuda())
        outs.append(torch.empty(shape, dtype=dt, device="cuda"))
        refs.append(torch.empty(shape, dtype=dt, device="cuda"))
    torch.cuda.synchronize()
    for rep in range(3):  # eager, captured, replayed
        chirp.chirp_batch_run(plans, xs, outs, bes)
        torch.cuda.synchronize()
    for pl, x, r, be in zip(plans, xs, refs, bes):
        (pl.chirpolator if be == 0 else pl.chimageator)(x, r)
    torch.cuda.synchronize()
    for i, (sc, pl, o, r, be) in enumerate(zip(scs, plans, outs, refs, bes)):
        assert torch.equal(o, r), i
        pl.status()
        x = xs[i].cpu().numpy()
        if be == 0:
            Vo = orc.chirpolator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len)
            assert vis_error(o.cpu().numpy(), Vo, sc.n_ant) < TOL_VIS, i
        else:
            Po = orc.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len,
                                 sc.xyz, sc.pix_lm)
            assert pow_error(o.cpu().numpy(), Po) < TOL_POW, i


@pytest.mark.parametrize("fft_row", [256, 512, 1024, 2048, 4096])
def test_forced_fft_split_matches_oracle(fft_row, k_dm):
    sc = _small(N=1 << 17, n_dm=3, nfft_min=1 << 15)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, fft_row=fft_row)
    for nfft, n_col, n_row in plan.fft_split():
        assert n_col * n_row == nfft
        if 16 <= nfft // fft_row <= 4096:
            assert n_row == fft_row
    V = np.empty((len(sc.dms), plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, V)
    Vo = orc.chirpolator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len)
    assert vis_error(V, Vo, sc.n_ant) < TOL_VIS


def test_autotuned_split_matches_oracle_and_is_cached(k_dm):
    sc = _beams(M=6, N=1 << 18, n_dm=3, nfft_min=1 << 16, n_side=4)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, flags=chirp.FLAG_AUTOTUNE)
    split = plan.fft_split()
    for nfft, n_col, n_row in split:
        assert n_col * n_row == nfft and 16 <= n_col <= 4096 and 256 <= n_row <= 4096
    again = chirp.Plan.from_scenario(sc, flags=chirp.FLAG_AUTOTUNE)
    assert again.fft_split() == split
    P = np.empty((len(sc.dms), plan.n_dump, plan.n_pix), np.float32)
    plan.chimageator(x, P)
    Po = orc.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len, sc.xyz,
                         sc.pix_lm)
    assert pow_error(P, Po) < TOL_POW


@pytest.mark.parametrize("mode", [chirp.BEAM_VIS, chirp.BEAM_TC_3XBF16])
def test_lean_plan_equals_full_plan_bit_for_bit(mode):
    """CHIRP_FLAG_LEAN holds one FFT-length group's spectra at a time (formed
    right before the group's DMs) and allocates the dedispersed-voltage buffer
    only when a search needs it: every entry point gives the default plan's
    outputs bit for bit, with less device memory.  Four DMs over three
    FFT-length groups, visited by the full, selective, Chirpolator, one-DM,
    true-delay and incoherent entry points in turn (so each run re-forms the
    spectra it needs)."""
    sc = _beams(N=1 << 17, n_dm=4)
    sc.dms = np.array([0.0, 6.0, 12.0, 40.0])
    kw = dict(beam_mode=mode, fb_chan=32, fb_int=8, fb_dm=sc.dms)
    full = chirp.Plan.from_scenario(sc, **kw)
    lean = chirp.Plan.from_scenario(sc, flags=chirp.FLAG_LEAN, **kw)
    assert len({full.dm_layout(d)["nfft"] for d in range(4)}) >= 3
    xd = torch.from_numpy(sc.voltages()).cuda()
    shp = (4, full.n_dump, full.n_pix)
    outs = {}
    for name, pl in (("full", full), ("lean", lean)):
        P = torch.empty(shp, dtype=torch.float32, device="cuda")
        pl.chimageator(xd, P)
        mask = np.zeros((4, pl.n_dump), np.uint8)
        mask[1, 20:30] = 1
        mask[3, 30:33] = 1
        S = torch.empty_like(P)
        pl.chimageator_selective(xd, mask, S)
        V = torch.empty((4, pl.n_dump, pl.n_pair), dtype=torch.complex64, device="cuda")
        pl.chirpolator(xd, V)
        y = torch.empty((sc.n_ant, sc.n_samp), dtype=torch.complex64, device="cuda")
        pl.dedisperse(xd, 2, y)
        T = torch.empty_like(P)
        pl.truedelay(xd, T)
        D = torch.empty((4, pl.info["fb_samples"]), dtype=torch.float32, device="cuda")
        pl.incoherent(xd, D)
        P2 = torch.empty_like(P)
        pl.chimageator(xd, P2)  # after the other entry points changed the spectra buffer
        torch.cuda.synchronize()
        outs[name] = [t.cpu().numpy() for t in (P, S, V, y, D, P2)] + [T.cpu().numpy()]
    for a, b in zip(outs["full"][:6], outs["lean"][:6]):
        assert np.array_equal(a, b)
    # true-delay dump sums are atomic adds: equal to the FP32 roundings of their order
    tf, tl = outs["full"][6], outs["lean"][6]
    assert np.array_equal(tf == 0, tl == 0)
    assert np.abs(tf - tl).max() <= 1e-5 * np.abs(tf).max()
    assert np.array_equal(outs["lean"][0], outs["lean"][5])
    ql = lean.info["workspace_bytes"]
    qf = full.info["workspace_bytes"]
    assert ql < qf, (ql, qf)
