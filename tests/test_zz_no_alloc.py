"""The allocation-free dedispersion entry point, for callers that cannot
allocate device memory (inside another library's stream capture, under a
memory budget reserved at start-up, or where cudaMalloc's implicit
synchronisation is not allowed).  Two calls in a row, with different shapes
and DMs, must each agree with chirp_dedisperse_run on a one-DM plan within
the FP32 voltage tolerance and with the FP64 oracle's dedispersion
(Sec. 2.3.2) within the same tolerance; the shared scratch must not leak
state from one call into the next; a warm call must leave the device's free
memory unchanged; host buffers and shapes beyond the fixed scratch are
refused clearly.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1109_3186_gb300 as chirp
from paper_1109_3186_gb300 import skymodel
from parity_util import TOL_Y_MAX, TOL_Y_RMS, y_error

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _reference(xd, f0, bw, dm, nfft_min, k_dm):
    M, N = xd.shape
    plan = chirp.Plan(np.zeros((M, 3)), f0, bw, N, [dm], 256, nfft_min, k_dm=k_dm)
    y = torch.empty((M, N), dtype=torch.complex64, device="cuda")
    plan.dedisperse(xd, 0, y)
    torch.cuda.synchronize()
    out = y.cpu().numpy()
    plan.close()
    return out


def test_noalloc_matches_plan_entry_point_and_oracle_on_two_calls(k_dm):
    f0, bw = 1.4e9, 8e6
    cases = [(3, 200000, 40.0, 1 << 14, 1), (5, 150000, 12.0, 1 << 13, 2)]
    for M, N, dm, nfft_min, seed in cases:
        x = skymodel.noise(M, N, seed)
        xd = torch.from_numpy(x).cuda()
        ref = _reference(xd, f0, bw, dm, nfft_min, k_dm)
        y = torch.full((M, N), complex(7.0, -7.0), dtype=torch.complex64, device="cuda")
        chirp.chirp_dedisperse_noalloc(xd, f0, bw, k_dm, dm, nfft_min, y)
        torch.cuda.synchronize()
        got = y.cpu().numpy()
        assert np.all(got[ref == 0] == 0)
        rms, mx = y_error(got, ref.astype(np.complex128))
        assert rms < TOL_Y_RMS and mx < TOL_Y_MAX, (M, N, dm, rms, mx)
        # the FP64 oracle of a one-DM search over the same samples
        yo = oracle.dedisperse(x, f0, bw, k_dm, [dm], 0, nfft_min)
        assert np.array_equal(got == 0, yo == 0)
        rms, mx = y_error(got, yo)
        assert rms < TOL_Y_RMS and mx < TOL_Y_MAX, ("oracle", M, N, dm, rms, mx)
        assert chirp.chirp_last_error() == ""


def test_noalloc_leaves_free_device_memory_unchanged(k_dm):
    M, N = 4, 120000
    xd = torch.from_numpy(skymodel.noise(M, N, 5)).cuda()
    y = torch.empty_like(xd)
    chirp.chirp_dedisperse_noalloc(xd, 1.4e9, 8e6, k_dm, 20.0, 1 << 14, y)  # set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for dm in (5.0, 30.0):
        chirp.chirp_dedisperse_noalloc(xd, 1.4e9, 8e6, k_dm, dm, 1 << 14, y)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_refuses_host_buffers_through_the_c_abi(k_dm):
    M, N = 2, 4096
    xd = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
    host = np.zeros((M, N), np.complex64)
    lib = chirp.load()
    rc = lib.chirp_dedisperse_noalloc(ctypes.c_void_p(host.ctypes.data), M, N, 1.4e9, 8e6, k_dm,
                                      10.0, 1 << 12, ctypes.c_void_p(xd.data_ptr()), None)
    assert rc == -1
    assert "device" in chirp.chirp_last_error()
    rc = lib.chirp_dedisperse_noalloc(ctypes.c_void_p(xd.data_ptr()), M, N, 1.4e9, 8e6, k_dm,
                                      10.0, 1 << 12, ctypes.c_void_p(host.ctypes.data), None)
    assert rc == -1


def test_noalloc_refuses_shapes_beyond_its_scratch(k_dm):
    x = torch.zeros((16, 1 << 20), dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(chirp.ChirpError) as ei:
        chirp.chirp_dedisperse_noalloc(x, 1.4e9, 8e6, k_dm, 50.0, 1 << 16, y)
    assert ei.value.code == -1
    assert "scratch" in str(ei.value)
