"""Batched back-ends of a row-pass chunk.

A full search inverse-transforms up to four DMs of an FFT-length group in one
row pass.  When their back-end is the staged CUDA-core correlator (the
Chirpolator in FP32, or the Chimageator's beams from visibilities), the column
passes write each DM's voltages into a slot of its own and one launch
correlates all of them (grid dimension z = DM), followed by one launch of the
beams from visibilities.  A lean plan keeps one voltage slot and runs the
per-DM back-ends.  The two must agree bit for bit -- the batched kernels do
each DM's arithmetic in the same order -- and the correlate stage must count
one launch per chunk instead of one per DM.
"""
import numpy as np
import pytest

import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _scene(M=12, n_dm=9, seed=4100):
    # DMs 0-40 over 8 MHz: most DMs share the 2^15 group, ragged dump ranges
    return skymodel.chimageator_medium(n_samp=1 << 18, n_dm=n_dm, n_ant=M, dm_max=40.0,
                                       nfft_min=1 << 15, dump_len=2048, bw=8e6, n_side=6,
                                       n_pulse=1, seed=seed)


def _chunks(plan, n_dm, dms=None):
    """Row-pass chunks of the full search (or of a search over the DMs dms):
    per FFT-length group, its DMs with a valid dump taken dm_chunk at a time."""
    first, last = plan.dump_range()
    groups = {}
    for d in range(n_dm) if dms is None else dms:
        if last[d] >= first[d]:
            groups.setdefault(plan.dm_layout(int(d))["nfft"], []).append(d)
    k = plan.info["dm_chunk"]
    return sum((len(v) + k - 1) // k for v in groups.values()), \
        sum(len(v) for v in groups.values())


def _correlate_launches(plan, fn):
    plan.stage_timing(True, stages=["correlate"])
    fn()
    return plan.stage_timing(False)["correlate"][1]


def _pair(sc, **kw):
    full = chirp.Plan.from_scenario(sc, **kw)
    lean = chirp.Plan.from_scenario(sc, flags=chirp.FLAG_LEAN, **kw)
    assert full.info["dm_chunk"] == 4
    return full, lean


def test_chirpolator_batched_equals_per_dm():
    sc = _scene(M=6)
    full, lean = _pair(sc, corr_mode=chirp.CORR_FP32_SIMT)
    n_chunk, n_valid = _chunks(full, len(sc.dms))
    assert n_chunk < n_valid
    xd = torch.from_numpy(sc.voltages()).cuda()
    shp = (len(sc.dms), full.n_dump, full.n_pair)
    out = {}
    for name, pl in (("full", full), ("lean", lean)):
        V = torch.full(shp, 3 + 3j, dtype=torch.complex64, device="cuda")
        n = _correlate_launches(pl, lambda: pl.chirpolator(xd, V))
        assert n == (n_chunk if name == "full" else n_valid), (name, n)
        out[name] = V.cpu()
    assert torch.equal(out["full"], out["lean"])


@pytest.mark.parametrize("M", [12, 20])
@pytest.mark.parametrize("mode", [chirp.BEAM_VIS, chirp.BEAM_VIS_BF16])
def test_visibility_beams_batched_equal_per_dm(M, mode):
    """12 antennas: the single-block correlator; 20: 12-antenna blocks and the
    block pair, both batched."""
    sc = _scene(M=M, seed=4200 + M)
    full, lean = _pair(sc, beam_mode=mode)
    n_chunk, n_valid = _chunks(full, len(sc.dms))
    xd = torch.from_numpy(sc.voltages()).cuda()
    shp = (len(sc.dms), full.n_dump, full.n_pix)
    out = {}
    for name, pl in (("full", full), ("lean", lean)):
        P = torch.full(shp, -1.0, dtype=torch.float32, device="cuda")
        n = _correlate_launches(pl, lambda: pl.chimageator(xd, P))
        assert n == (n_chunk if name == "full" else n_valid), (name, n)
        out[name] = P.cpu()
    assert torch.equal(out["full"], out["lean"])


def test_dense_selection_batched_with_dump_lists():
    """A selection dense enough for the multi-DM inverse: the batched
    back-ends take each DM's dump list; selected cells equal the full
    search, all others are zero."""
    sc = _scene(seed=4300)
    full, lean = _pair(sc, beam_mode=chirp.BEAM_VIS)
    xd = torch.from_numpy(sc.voltages()).cuda()
    shp = (len(sc.dms), full.n_dump, full.n_pix)
    ref = torch.empty(shp, dtype=torch.float32, device="cuda")
    full.chimageator(xd, ref)
    first, last = full.dump_range()
    rng = np.random.default_rng(7)
    mask = (rng.random((len(sc.dms), full.n_dump)) < 0.5).astype(np.uint8)
    pick = np.zeros(mask.shape, bool)
    for d in range(len(sc.dms)):
        pick[d, first[d]:last[d] + 1] = mask[d, first[d]:last[d] + 1] > 0
    out = {}
    for name, pl in (("full", full), ("lean", lean)):
        S = torch.full(shp, 5.0, dtype=torch.float32, device="cuda")
        pl.chimageator_selective(xd, mask, S)
        out[name] = S.cpu()
    assert torch.equal(out["full"], out["lean"])
    r = ref.cpu().numpy()
    s = out["full"].numpy()
    assert np.array_equal(s[pick], r[pick])
    assert np.all(s[~pick] == 0)


@pytest.mark.parametrize("mode", [chirp.BEAM_VIS, chirp.BEAM_TC_3XBF16])
def test_run_selection_chunks_share_row_passes(mode):
    """Runs of a few dumps per DM: each group's DMs go through one row pass
    over their own listed blocks per chunk, then the column passes and the
    back-ends (batched in the visibility form, one DM after another for the
    tensor-core beams); the full plan, the lean plan and the full search agree
    bit for bit on the selected cells, all other cells are zero."""
    sc = _scene(seed=4400)
    full, lean = _pair(sc, beam_mode=mode)
    xd = torch.from_numpy(sc.voltages()).cuda()
    shp = (len(sc.dms), full.n_dump, full.n_pix)
    ref = torch.empty(shp, dtype=torch.float32, device="cuda")
    full.chimageator(xd, ref)
    first, last = full.dump_range()
    mask = np.zeros((len(sc.dms), full.n_dump), np.uint8)
    rng = np.random.default_rng(9)
    for d in range(len(sc.dms)):
        if last[d] - first[d] > 8:
            m0 = int(rng.integers(first[d], last[d] - 4))
            mask[d, m0:m0 + 3] = 1
    pick = mask.astype(bool)
    out = {}
    for name, pl in (("full", full), ("lean", lean)):
        S = torch.full(shp, 5.0, dtype=torch.float32, device="cuda")
        pl.stage_timing(True, stages=["inv_rows"])
        pl.chimageator_selective(xd, mask, S)
        n_rows = pl.stage_timing(False)["inv_rows"][1]
        n_chunk, n_sel = _chunks(pl, len(sc.dms), np.nonzero(pick.any(axis=1))[0])
        assert n_rows == n_chunk < n_sel, (name, n_rows, n_chunk)
        out[name] = S.cpu()
    assert torch.equal(out["full"], out["lean"])
    s = out["full"].numpy()
    assert np.array_equal(s[pick], ref.cpu().numpy()[pick])
    assert np.all(s[~pick] == 0)
