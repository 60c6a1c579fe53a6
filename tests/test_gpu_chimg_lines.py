"""The partial-sum recursion of the Chimageator's imaging step on the GPU
(chirp_chimg_lines_run, App. B.2.1): one cumulative trajectory sum per
(line, window start) gives every trial of the line, in the paper's own model
of Sec. 4.2.  Checked element by element against the FP64 oracle's images of
the same trials, each from its own taps (oracle.chimg.paper_image_direct), on
the Y the library's own gridding pass writes from voltages holding noise and
perfect chirps of two of the trials; incomplete windows are exactly zero, the
chirps' trials peak where their windows end, and bad trial lists or host
buffers are refused."""
import ctypes
import math

import numpy as np
import pytest

import paper_1109_3186_gb300 as chirp
from oracle import chimg as oc
from paper_1109_3186_gb300 import chimg as gc

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

B, L, NS, M, F, D = 8e6, 256, 16, 8, 1, 500.0


def _chirp(n_win, rate, start, n_samp):
    """A unit chirp of the paper's model (sweep 0..B over n_win dumps from
    dump `start`) as every antenna receives it (delays p tau)."""
    T = n_win * L / B
    fdot = B / T
    tau = rate / fdot
    y = np.zeros((M, n_samp), np.complex128)
    t = np.arange(n_win * L) / B
    y[:, start * L:(start + n_win) * L] = np.exp(
        1j * math.pi * fdot * (t[None, :] - np.arange(M)[:, None] * tau) ** 2)
    return y


def test_lines_match_the_oracle_trial_by_trial():
    n_dump = 40
    n_samp = n_dump * L
    rates = [0.2 * B / (NS * L), -0.35 * B / (NS * L), 0.6 * B / (NS * L)]
    lens = [[3, 6, 11], [4, 9], [2, 5, 8, 16]]
    rng = np.random.default_rng(31)
    y = (rng.standard_normal((M, n_samp)) + 1j * rng.standard_normal((M, n_samp))) * 0.4
    y += _chirp(11, rates[0], 7, n_samp) + _chirp(8, rates[2], 20, n_samp)
    plan = gc.ChimgPlan(M, D, 1.4e9, B, n_samp, [10.0], L, [0.0], NS, half_width=F)
    Yd = torch.empty((n_dump, NS), dtype=torch.complex64, device="cuda")
    plan.grid(torch.from_numpy(y.astype(np.complex64)).cuda(), Yd)
    E = gc.lines_run(Yd, M, NS, L, B, F, rates, lens).cpu().numpy()
    Yo = Yd.cpu().numpy().astype(np.complex128).T            # [Ns][n_dump]
    t = 0
    for g, rate in enumerate(rates):
        Eo = oc.paper_image_direct(Yo, M, rate, lens[g], B, L, NS, F)
        for i, nw in enumerate(lens[g]):
            got, ref = E[t], Eo[i]
            assert np.all(got[:nw - 1] == 0)
            scale = ref.max()
            assert np.abs(got - ref).max() <= 1e-5 * scale, (g, nw)
            big = ref > 1e-3 * scale
            assert np.max(np.abs(got - ref)[big] / ref[big]) <= 1e-3, (g, nw)
            t += 1
    # the chirps' own trials peak where their windows end
    assert int(np.argmax(E[2])) == 7 + 11 - 1
    assert int(np.argmax(E[5 + 2])) == 20 + 8 - 1


def test_refuses_bad_trial_lists_and_host_buffers():
    Yd = torch.zeros((8, NS), dtype=torch.complex64, device="cuda")
    with pytest.raises(chirp.ChirpError):
        gc.lines_run(Yd, M, NS, L, B, F, [1.0], [[]])
    lib = chirp.load()
    rate = (ctypes.c_double * 1)(1.0)
    off = (ctypes.c_int * 2)(0, 2)
    bad = (ctypes.c_int * 2)(5, 3)                            # not ascending
    E = torch.zeros((2, 8), dtype=torch.float32, device="cuda")
    rc = lib.chirp_chimg_lines_run(ctypes.c_void_p(Yd.data_ptr()), 8, M, NS, L, B, F, rate, 1, off,
                                   bad, ctypes.c_void_p(E.data_ptr()), None)
    assert rc == chirp.CHIRP_EINVAL
    host = np.zeros((8, NS), np.complex64)
    good = (ctypes.c_int * 2)(3, 5)
    rc = lib.chirp_chimg_lines_run(ctypes.c_void_p(host.ctypes.data), 8, M, NS, L, B, F, rate, 1,
                                   off, good, ctypes.c_void_p(E.data_ptr()), None)
    assert rc == chirp.CHIRP_EINVAL
