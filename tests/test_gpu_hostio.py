"""Host buffers through the search entry points.

Page-locked (pinned) host input is copied in time chunks while the forward
transforms follow it, and page-locked host output goes back one DM slab at a
time while later DMs are searched.  Each of these paths must give, bit for
bit, what the same plan computes from device buffers:
- the Chimageator and the Chirpolator, with pinned or pageable host buffers
  on either side, and complex int8 input;
- lean plans (spectra formed per group);
- back-to-back calls from two pinned inputs into device outputs with no
  synchronisation in between: the second call's input copy must not
  overwrite the staging buffer while the first search still reads it.
"""
import numpy as np
import pytest

import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _beams(seed=1002, N=1 << 18, n_dm=5, M=8):
    # DMs 0-150 over 8 MHz: sweeps of up to ~29k samples, so several
    # FFT-length groups whose blocks an input time chunk covers only in part
    return skymodel.chimageator_medium(n_samp=N, n_dm=n_dm, n_ant=M, dm_max=150.0,
                                       nfft_min=1 << 14, dump_len=2048, bw=8e6, n_side=8,
                                       n_pulse=1, seed=seed)


def _pinned(a: np.ndarray):
    return torch.from_numpy(a).pin_memory()


@pytest.mark.parametrize("inp", ["pinned", "pageable"])
@pytest.mark.parametrize("out", ["pinned", "pageable", "device"])
def test_chimageator_host_paths_equal_device_path(inp, out):
    sc = _beams()
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc)
    assert plan.info["n_group"] >= 2
    shape = (len(sc.dms), plan.n_dump, plan.n_pix)
    ref = torch.empty(shape, dtype=torch.float32, device="cuda")
    plan.chimageator(torch.from_numpy(x).cuda(), ref)
    xin = _pinned(x) if inp == "pinned" else x
    if out == "device":
        P = torch.full(shape, -1.0, dtype=torch.float32, device="cuda")
    elif out == "pinned":
        P = torch.full(shape, -1.0, dtype=torch.float32).pin_memory()
    else:
        P = np.full(shape, -1.0, np.float32)
    for _ in range(2):  # twice: the staging buffers are reused
        plan.chimageator(xin, P)
        torch.cuda.synchronize()
        got = P.cpu() if isinstance(P, torch.Tensor) else torch.from_numpy(P)
        assert torch.equal(got, ref.cpu())


def test_chirpolator_pinned_host_equals_device():
    sc = _beams(seed=7, n_dm=4, M=6)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc)
    shape = (len(sc.dms), plan.n_dump, plan.n_pair)
    ref = torch.empty(shape, dtype=torch.complex64, device="cuda")
    plan.chirpolator(torch.from_numpy(x).cuda(), ref)
    V = torch.zeros(shape, dtype=torch.complex64).pin_memory()
    plan.chirpolator(_pinned(x), V)
    assert torch.equal(V, ref.cpu())


def test_int8_pinned_input_equals_device_input():
    sc = _beams(seed=11, n_dm=3)
    q, scale = skymodel.quantize_ci8(sc.voltages())
    plan = chirp.Plan.from_scenario(sc, in_type=chirp.IN_CI8, in_scale=scale)
    shape = (len(sc.dms), plan.n_dump, plan.n_pix)
    ref = torch.empty(shape, dtype=torch.float32, device="cuda")
    plan.chimageator(torch.from_numpy(q).cuda(), ref)
    P = torch.zeros(shape, dtype=torch.float32).pin_memory()
    plan.chimageator(_pinned(q), P)
    assert torch.equal(P, ref.cpu())


def test_lean_plan_pinned_buffers_equal_device_path():
    sc = _beams(seed=13)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc, flags=chirp.FLAG_LEAN)
    shape = (len(sc.dms), plan.n_dump, plan.n_pix)
    ref = torch.empty(shape, dtype=torch.float32, device="cuda")
    plan.chimageator(torch.from_numpy(x).cuda(), ref)
    P = torch.zeros(shape, dtype=torch.float32).pin_memory()
    plan.chimageator(_pinned(x), P)
    assert torch.equal(P, ref.cpu())


def test_back_to_back_pinned_inputs_do_not_race_on_the_staging_buffer():
    sc1, sc2 = _beams(seed=21), _beams(seed=22)
    x1, x2 = sc1.voltages(), sc2.voltages()
    plan = chirp.Plan.from_scenario(sc1)
    shape = (len(sc1.dms), plan.n_dump, plan.n_pix)
    r1 = torch.empty(shape, dtype=torch.float32, device="cuda")
    r2 = torch.empty_like(r1)
    plan.chimageator(torch.from_numpy(x1).cuda(), r1)
    plan.chimageator(torch.from_numpy(x2).cuda(), r2)
    torch.cuda.synchronize()
    assert not torch.equal(r1, r2)
    h1, h2 = _pinned(x1), _pinned(x2)
    for _ in range(3):
        P1 = torch.empty_like(r1)
        P2 = torch.empty_like(r1)
        plan.chimageator(h1, P1)   # returns with the search still running
        plan.chimageator(h2, P2)
        torch.cuda.synchronize()
        assert torch.equal(P1, r1)
        assert torch.equal(P2, r2)
