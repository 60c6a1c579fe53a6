"""Parity at the full sizes of the two plain-FP32 workloads, in the launch
configuration the benchmark times (same scenario recipe and seed, same plan
options, the current torch stream, device-resident input).  The GPU computes
the whole search; the FP64 oracle recomputes sampled cells one by one, and
properties that hold at any size are checked on the whole output.

- Chimageator (the library's AUTO choice and the split-BF16 tensor-core
  form): 12 antennas within 6 km, 32 MHz at 1.4 GHz, 2^22 samples,
  64 DMs in 0-300, FFT >= 2^18 (four FFT-length groups), 32 x 32 beams over
  1 deg, dumps of 4096.  Sampled: DM 0 and the first and last DM of every
  group, each at its first valid dumps, a middle dump and its last valid
  dumps, plus the dump of every injected burst at its nearest trial DM; all
  1024 beams.  Whole output: zero outside each DM's valid dumps, positive
  inside.
- Chirpolator: 6 antennas within 2 km, 8 MHz, 2^20 samples, 16 DMs in
  0-150, FFT 2^16, dumps of 1024.  Four DMs (DM 0, the two around the
  burst's DM 75, DM 150) in full against the oracle; whole output: zero
  outside the valid dumps, autocorrelations positive (and real to 1e-5) inside,
  |V_pq|^2 <= V_pp V_qq (Cauchy-Schwarz for every dump).
Tolerances: the FP32 budget, 1e-5 relative on powers and visibilities.
"""
import numpy as np
import pytest

import oracle as orc
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_POW, TOL_VIS, pair_index, pow_error, vis_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("mode,resolved", [(chirp.BEAM_AUTO, chirp.BEAM_VIS),
                                           (chirp.BEAM_TC_3XBF16, chirp.BEAM_TC_3XBF16)])
def test_chimageator_full_size_sampled_cells(mode, resolved):
    """The benchmark's headline form (AUTO: the visibility identity, the
    faster exact form here) and the split-BF16 tensor-core GEMM."""
    sc = skymodel.chimageator_medium(seed=1002)      # the benchmark's observation
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, beam_mode=mode, stream=torch.cuda.current_stream())
    assert plan.info["beam_mode"] == resolved
    xd = torch.from_numpy(x).cuda()
    P = torch.empty((len(sc.dms), plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    plan.chimageator(xd, P)
    plan.status()
    first, last = plan.dump_range()
    del xd

    # whole output: zeros outside each DM's valid dumps, positive powers inside
    idx = torch.arange(plan.n_dump, device="cuda")[None, :]
    f_t = torch.from_numpy(np.asarray(first)).cuda()[:, None]
    l_t = torch.from_numpy(np.asarray(last)).cuda()[:, None]
    inside = (idx >= f_t) & (idx <= l_t)
    assert torch.all(P[~inside] == 0)
    assert torch.all(P[inside] > 0)

    groups = {}
    for d in range(len(sc.dms)):
        groups.setdefault(plan.dm_layout(d)["nfft"], []).append(d)
    assert len(groups) == 4
    dms = sorted({0} | {g[0] for g in groups.values()} | {g[-1] for g in groups.values()})
    cells = []                                       # (DM number, m0, m1)
    for d in dms:
        f, l = first[d], last[d]
        mid = (f + l) // 2
        cells += [(d, f, f + 2), (d, mid, mid + 1), (d, l - 1, l + 1)]
    for p in sc.pulses:
        d = int(np.argmin(np.abs(sc.dms - p.dm)))
        m = int(p.t0 // sc.dump_len)
        if first[d] <= m <= last[d]:
            cells.append((d, m, m + 1))
    x128 = x.astype(np.complex128)
    for d, m0, m1 in cells:
        Po = orc.chimageator(x128, sc.f0, sc.bw, sc.k_dm, sc.dms, sc.nfft_min, sc.dump_len,
                             sc.xyz, sc.pix_lm, d_sel=[d], m0=m0, m1=m1)[0]
        Pg = P[d, m0:m1].cpu().numpy()
        err = pow_error(Pg, Po)
        assert err < TOL_POW, (d, m0, m1, err)
    assert len(cells) >= 24
    plan.close()


def test_chirpolator_full_size():
    sc = skymodel.chirpolator_small()                # 6 ant, 2^20 samples, 16 DMs, FFT 2^16
    assert (sc.n_ant, sc.n_samp, len(sc.dms), sc.nfft_min, sc.dump_len) == (6, 1 << 20, 16,
                                                                             1 << 16, 1024)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, stream=torch.cuda.current_stream())
    xd = torch.from_numpy(x).cuda()
    V = torch.empty((len(sc.dms), plan.n_dump, plan.n_pair), dtype=torch.complex64,
                    device="cuda")
    plan.chirpolator(xd, V)
    plan.status()
    Vg = V.cpu().numpy()
    first, last = plan.dump_range()

    pairs = pair_index(sc.n_ant)
    autos = [pairs.index((a, a)) for a in range(sc.n_ant)]
    for d in range(len(sc.dms)):
        assert np.all(Vg[d, :first[d]] == 0) and np.all(Vg[d, last[d] + 1:] == 0)
        v = Vg[d, first[d]:last[d] + 1].astype(np.complex128)
        a = v[:, autos]
        assert np.all(a.real > 0) and np.all(np.abs(a.imag) <= 1e-5 * a.real)
        for k, (p, q) in enumerate(pairs):
            bound = a[:, p].real * a[:, q].real
            assert np.all(np.abs(v[:, k]) ** 2 <= bound * (1 + 1e-5))

    p_dm = sc.pulses[0].dm
    near = np.argsort(np.abs(sc.dms - p_dm))[:2]
    sel = sorted({0, int(near[0]), int(near[1]), len(sc.dms) - 1})
    Vo = orc.chirpolator(x, sc.f0, sc.bw, sc.k_dm, sc.dms, sc.nfft_min, sc.dump_len, d_sel=sel)
    for i, d in enumerate(sel):
        err = vis_error(Vg[d, first[d]:last[d] + 1], Vo[i, first[d]:last[d] + 1], sc.n_ant)
        assert err < TOL_VIS, (d, err)
    plan.close()
