"""Failure detection without a GPU fault.

- The device watchdog: the bounded mbarrier wait that every producer and
  consumer role of the tensor-core kernels uses, run on a barrier that
  nothing arrives at, gives up after its poll limit and raises the error
  word the host reads (CHIRP_ETIMEOUT); the context stays usable and a
  search afterwards still matches the oracle.
- Host-side injection: a plan larger than the device's memory is refused
  with CHIRP_ENOMEM (no partial plan is left behind), and the next plan
  works.
"""
import numpy as np
import pytest

import oracle as orc
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_VIS, vis_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _small_search_matches_oracle(k_dm):
    sc = skymodel.chirpolator_small(n_samp=1 << 15, n_dm=2, dm_max=20.0, nfft_min=1 << 12)
    x = sc.voltages()
    plan = chirp.Plan.from_scenario(sc)
    V = np.empty((2, plan.n_dump, plan.n_pair), np.complex64)
    plan.chirpolator(x, V)
    plan.status()  # raises if a device wait gave up
    Vo = orc.chirpolator(x, sc.f0, sc.bw, k_dm, sc.dms, sc.nfft_min, sc.dump_len)
    assert vis_error(V, Vo, sc.n_ant) < TOL_VIS
    plan.close()


def test_watchdog_gives_up_and_the_context_stays_usable(k_dm):
    for polls in (64, 1 << 12, 1 << 16):
        rc, ms = chirp.chirp_watchdog_selftest(polls)
        assert rc == chirp.CHIRP_ETIMEOUT, (polls, rc, chirp.chirp_last_error())
        assert 0.0 < ms < 2000.0
    _small_search_matches_oracle(k_dm)


def test_plan_larger_than_the_device_is_refused_cleanly(k_dm):
    free, total = torch.cuda.mem_get_info()
    # 64 antennas x 2^32 samples: the voltage and spectrum workspaces alone
    # need ~2 x 2.2 TB
    xyz = skymodel.antenna_positions(64, 6000.0, 5)
    assert 64 * (1 << 32) * 8 > 2 * total
    with pytest.raises(chirp.ChirpError) as e:
        chirp.Plan(xyz, 1.4e9, 32e6, 1 << 32, [0.0], 4096, 1 << 24)
    assert e.value.code == chirp.CHIRP_ENOMEM, str(e.value)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free - (64 << 20)  # nothing left allocated
    _small_search_matches_oracle(k_dm)
