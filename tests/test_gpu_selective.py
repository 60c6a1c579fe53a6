"""The selective coherent search computes, in the selected (DM, dump) cells,
what the full search computes there, and zeros elsewhere.  An FFT-length
group whose selected DMs need most of their overlap-save blocks (scattered
cells) runs the full multi-DM inverse and restricts the back-end to the
selected dumps; a group that needs few blocks (runs of dumps) is inverse
transformed one DM at a time over its listed blocks.  The tests check which
of the two ran (row-pass launch counts) and, through the bit-for-bit
equality of the visibilities, also pin the multi-DM row pass to the
single-DM one."""
import numpy as np
import pytest

import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("mode", [chirp.BEAM_VIS, chirp.BEAM_TC_3XBF16, chirp.BEAM_FP32_SIMT])
def test_selective_beams_equal_full_on_selected_cells(mode):
    sc = skymodel.chimageator_medium(n_samp=1 << 18, n_dm=6, n_ant=12, dm_max=150.0,
                                     nfft_min=1 << 15, dump_len=2048, n_side=8, n_pulse=1)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, beam_mode=mode)
    xd = torch.from_numpy(x).cuda()
    full = torch.empty((6, plan.n_dump, plan.n_pix), dtype=torch.float32, device="cuda")
    plan.chimageator(xd, full)
    rng = np.random.default_rng(3)
    mask = (rng.random((6, plan.n_dump)) < 0.15).astype(np.uint8)
    mask[2] = 0
    mask[4, 40:60] = 1
    sel = torch.empty_like(full)
    plan.chimageator_selective(xd, mask, sel)
    F, S = full.cpu().numpy(), sel.cpu().numpy()
    first, last = plan.dump_range()
    valid = np.zeros_like(mask, bool)
    for d in range(6):
        valid[d, first[d]:last[d] + 1] = True
    pick = (mask.astype(bool) & valid)
    assert np.all(S[~pick] == 0)
    assert pick.sum() > 20
    assert np.abs(S[pick] - F[pick]).max() <= 1e-6 * np.abs(F[pick]).max()


def test_selective_visibilities_equal_full():
    sc = skymodel.chirpolator_small(n_samp=1 << 18, n_dm=5, dm_max=100.0, nfft_min=1 << 15)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc)
    assert plan.info["dm_chunk"] >= 2
    assert len(set(plan.dm_layout(d)["nfft"] for d in range(5))) < 5  # a group holds 2+ DMs
    full = np.empty((5, plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, full)
    mask = np.zeros((5, plan.n_dump), np.uint8)
    mask[1, 10:12] = 1
    mask[3, 100:180] = 1
    mask[3, 240] = 1
    sel = np.empty_like(full)
    plan.chirpolator_selective(x, mask, sel)
    pick = mask.astype(bool)
    assert np.array_equal(sel[pick], full[pick])
    assert np.all(sel[~pick] == 0)


def _row_launches(plan, fn):
    """Inverse row-pass launches of one call of fn."""
    plan.stage_timing(True, stages=["inv_rows"])
    fn()
    return plan.stage_timing(False)["inv_rows"][1]


def _runs_mask(valid, seed, run=3):
    """One run of `run` dumps per DM inside its valid dumps: few blocks."""
    rng = np.random.default_rng(seed)
    mask = np.zeros(valid.shape, np.uint8)
    for d in range(valid.shape[0]):
        v = np.nonzero(valid[d])[0]
        if len(v) > run:
            m0 = int(v[0] + rng.integers(0, len(v) - run))
            mask[d, m0:m0 + run] = 1
    return mask


@pytest.mark.parametrize("frac", [0.3, 0.7, 1.0])
def test_scattered_selections_equal_full(frac):
    """Scattered cells need every block: the multi-DM inverse with a restricted
    back-end gives the full search's values bit for bit and zeros elsewhere."""
    sc = skymodel.chirpolator_small(n_samp=1 << 18, n_dm=5, dm_max=100.0, nfft_min=1 << 15)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc)
    full = np.empty((5, plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, full)
    first, last = plan.dump_range()
    valid = np.zeros((5, plan.n_dump), bool)
    for d in range(5):
        valid[d, first[d]:last[d] + 1] = True
    rng = np.random.default_rng(11)
    mask = (rng.random(valid.shape) < frac).astype(np.uint8)
    mask[0, first[0]:first[0] + 10] = 0
    sel = np.full_like(full, np.complex64(7 + 7j))
    n_rows = _row_launches(plan, lambda: plan.chirpolator_selective(x, mask, sel))
    n_sel_dms = int(np.sum((mask.astype(bool) & valid).any(axis=1)))
    assert n_rows < n_sel_dms  # row passes shared by the DMs of a group
    pick = mask.astype(bool) & valid
    assert np.array_equal(sel[pick], full[pick])
    assert np.all(sel[~pick] == 0)


def test_run_selections_equal_full_with_per_dm_blocks():
    """Runs of a few dumps need few blocks: per-DM block lists (the DMs of a
    group share a row-pass launch), the full search's values bit for bit there
    and zeros elsewhere; a search mixing a scattered group and a run-shaped
    one takes both paths at once."""
    sc = skymodel.chirpolator_small(n_samp=1 << 18, n_dm=5, dm_max=100.0, nfft_min=1 << 15)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc)
    full = np.empty((5, plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, full)
    first, last = plan.dump_range()
    valid = np.zeros((5, plan.n_dump), bool)
    for d in range(5):
        valid[d, first[d]:last[d] + 1] = True
    mask = _runs_mask(valid, 5)
    sel = np.full_like(full, np.complex64(7 + 7j))
    n_rows = _row_launches(plan, lambda: plan.chirpolator_selective(x, mask, sel))
    sel_dms = np.nonzero((mask.astype(bool) & valid).any(axis=1))[0]
    assert len(sel_dms) >= 4
    # one row pass per chunk of up to dm_chunk DMs of an FFT-length group,
    # each DM over its own listed blocks
    per_group = {}
    for d in sel_dms:
        per_group[plan.dm_layout(int(d))["nfft"]] = per_group.get(plan.dm_layout(int(d))["nfft"], 0) + 1
    k = plan.info["dm_chunk"]
    assert n_rows == sum((c + k - 1) // k for c in per_group.values())
    pick = mask.astype(bool) & valid
    assert np.array_equal(sel[pick], full[pick])
    assert np.all(sel[~pick] == 0)
    # mixed: the largest group's DMs scattered, the others in runs
    nf = [plan.dm_layout(d)["nfft"] for d in range(5)]
    big = [d for d in range(5) if nf[d] == max(nf)]
    rng = np.random.default_rng(12)
    for d in big:
        mask[d] = (rng.random(plan.n_dump) < 0.5).astype(np.uint8)
    sel[:] = np.complex64(7 + 7j)
    plan.chirpolator_selective(x, mask, sel)
    pick = mask.astype(bool) & valid
    assert np.array_equal(sel[pick], full[pick])
    assert np.all(sel[~pick] == 0)


# ---------------------------------------------------------------- vs the oracle
# The selected cells are checked directly against the FP64 oracle's full search
# (Sec. 2.3.2 dedispersion, Eq. xpq visibilities, Sec. 2.4.2 phased beams), so a
# fault shared by the full and the selective GPU paths, or a DM/dump indexing
# fault that only the selective lists have, cannot pass.  Scattered selections
# (30 % and 95 % of the cells) take the multi-DM inverse with dump lists in the
# back-end; run-shaped selections take the per-DM block lists.
from parity_util import TOL_POW, TOL_VIS, pow_error, vis_error  # noqa: E402

import oracle  # noqa: E402

_BEAMS = dict(n_samp=1 << 18, n_dm=6, n_ant=12, dm_max=150.0, nfft_min=1 << 15, dump_len=2048,
              n_side=8, n_pulse=1)
_VIS = dict(n_samp=1 << 18, n_dm=5, dm_max=100.0, nfft_min=1 << 15)


def _valid(plan, n_dm):
    first, last = plan.dump_range()
    v = np.zeros((n_dm, plan.n_dump), bool)
    for d in range(n_dm):
        v[d, first[d]:last[d] + 1] = True
    return v


def _mask(valid, kind, seed):
    if kind == "runs":
        return _runs_mask(valid, seed, run=6)
    rng = np.random.default_rng(seed)
    return (rng.random(valid.shape) < kind).astype(np.uint8)


@pytest.fixture(scope="module")
def beam_case(k_dm):
    sc = skymodel.chimageator_medium(**_BEAMS)
    x = sc.voltages()
    P = oracle.chimageator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len, sc.xyz,
                           sc.pix_lm)
    return sc, x, P


@pytest.fixture(scope="module")
def vis_case(k_dm):
    sc = skymodel.chirpolator_small(**_VIS)
    x = sc.voltages()
    V = oracle.chirpolator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len)
    return sc, x, V


@pytest.mark.parametrize("frac", [0.3, 0.95, "runs"])
@pytest.mark.parametrize("mode", [chirp.BEAM_AUTO, chirp.BEAM_VIS, chirp.BEAM_TC_3XBF16,
                                  chirp.BEAM_FP32_SIMT])
def test_selective_beams_match_oracle(beam_case, mode, frac):
    sc, x, Po = beam_case
    n_dm = len(sc.dms)
    plan = chirp.Plan.from_scenario(sc, beam_mode=mode)
    valid = _valid(plan, n_dm)
    mask = _mask(valid, frac, 40 if frac == "runs" else 40 + int(100 * frac))
    out = torch.full((n_dm, plan.n_dump, plan.n_pix), 5.0, dtype=torch.float32, device="cuda")
    plan.chimageator_selective(torch.from_numpy(x).cuda(), mask, out)
    S = out.cpu().numpy()
    plan.close()
    pick = mask.astype(bool) & valid
    assert pick.sum() > (12 if frac == "runs" else 20)
    assert np.all(S[~pick] == 0)
    err = pow_error(S[pick], Po[pick])
    assert err <= TOL_POW, (mode, frac, err)


@pytest.mark.parametrize("frac", [0.3, 0.95, "runs"])
def test_selective_visibilities_match_oracle(vis_case, frac):
    sc, x, Vo = vis_case
    n_dm = len(sc.dms)
    plan = chirp.Plan.from_scenario(sc)
    valid = _valid(plan, n_dm)
    mask = _mask(valid, frac, 70 if frac == "runs" else 70 + int(100 * frac))
    sel = np.full((n_dm, plan.n_dump, plan.n_pair), np.complex64(3 - 3j))
    plan.chirpolator_selective(x, mask, sel)
    plan.close()
    pick = mask.astype(bool) & valid
    assert np.all(sel[~pick] == 0)
    err = vis_error(sel[pick], Vo[pick], sc.n_ant)
    assert err <= TOL_VIS, (frac, err)
