"""The selective coherent search computes, in the selected (DM, dump) cells,
what the full search computes there, and zeros elsewhere.  The full search
runs the inverse row pass of several DMs of a group in one launch, the
selective search one DM at a time, so the bit-for-bit equality of the
visibilities also pins the multi-DM row pass to the single-DM one."""
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


@pytest.mark.parametrize("frac", [0.7, 0.9, 1.0])
def test_dense_selections_equal_full(frac):
    """Selections either side of the 80 % switch to the full multi-DM search
    (which then clears the unselected cells): both give the full search's
    values bit for bit and zeros elsewhere."""
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
    share = (mask.astype(bool) & valid).sum() / valid.sum()
    assert (share >= 0.8) == (frac >= 0.9)
    sel = np.full_like(full, np.complex64(7 + 7j))
    plan.chirpolator_selective(x, mask, sel)
    pick = mask.astype(bool) & valid
    assert np.array_equal(sel[pick], full[pick])
    assert np.all(sel[~pick] == 0)


# ---------------------------------------------------------------- vs the oracle
# The selected cells are checked directly against the FP64 oracle's full search
# (Sec. 2.3.2 dedispersion, Eq. xpq visibilities, Sec. 2.4.2 phased beams), so a
# fault shared by the full and the selective GPU paths, or a DM/dump indexing
# fault that only the selective lists have, cannot pass.  Selections either side
# of the 80 % switch cover both the per-DM block/dump lists and the full search
# that clears the unselected cells afterwards.
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


def _mask(valid, frac, seed):
    rng = np.random.default_rng(seed)
    mask = (rng.random(valid.shape) < frac).astype(np.uint8)
    share = (mask.astype(bool) & valid).sum() / valid.sum()
    assert (share >= 0.8) == (frac >= 0.9)
    return mask


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


@pytest.mark.parametrize("frac", [0.3, 0.95])
@pytest.mark.parametrize("mode", [chirp.BEAM_AUTO, chirp.BEAM_VIS, chirp.BEAM_TC_3XBF16,
                                  chirp.BEAM_FP32_SIMT])
def test_selective_beams_match_oracle(beam_case, mode, frac):
    sc, x, Po = beam_case
    n_dm = len(sc.dms)
    plan = chirp.Plan.from_scenario(sc, beam_mode=mode)
    valid = _valid(plan, n_dm)
    mask = _mask(valid, frac, 40 + int(100 * frac))
    out = torch.full((n_dm, plan.n_dump, plan.n_pix), 5.0, dtype=torch.float32, device="cuda")
    plan.chimageator_selective(torch.from_numpy(x).cuda(), mask, out)
    S = out.cpu().numpy()
    plan.close()
    pick = mask.astype(bool) & valid
    assert pick.sum() > 20
    assert np.all(S[~pick] == 0)
    err = pow_error(S[pick], Po[pick])
    assert err <= TOL_POW, (mode, frac, err)


@pytest.mark.parametrize("frac", [0.3, 0.95])
def test_selective_visibilities_match_oracle(vis_case, frac):
    sc, x, Vo = vis_case
    n_dm = len(sc.dms)
    plan = chirp.Plan.from_scenario(sc)
    valid = _valid(plan, n_dm)
    mask = _mask(valid, frac, 70 + int(100 * frac))
    sel = np.full((n_dm, plan.n_dump, plan.n_pair), np.complex64(3 - 3j))
    plan.chirpolator_selective(x, mask, sel)
    plan.close()
    pick = mask.astype(bool) & valid
    assert np.all(sel[~pick] == 0)
    err = vis_error(sel[pick], Vo[pick], sc.n_ant)
    assert err <= TOL_VIS, (frac, err)
