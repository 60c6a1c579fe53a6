"""Parity of the CUDA Chimageator pre-integrator on a uniform linear array
(chirp_chimg_*) with the FP64 oracle (oracle/chimg.py): the integrated
spatial spectra Y and the trajectory images E element by element, for 5 to
32 antennas, both weightings, F = 0..2 and a ragged tail; and a perfect
chirp found at its direction.

Tolerances: the GPU sums each dump's L products per spacing in FP32 before
the spatial DFT (the oracle transforms every sample), so Y agrees to a few
FP32 roundings of the dump's sum: 1e-5 of its largest magnitude.  E = |P|^2
sums (2F+1) n_win filter taps: 1e-4 of its largest value per DM, and entry
by entry above 1e-3 of that value REL_E_ABOVE_FLOOR relative."""
import math

import numpy as np
import pytest

from oracle import chimg as ochimg
from oracle import cpi as ocpi
from paper_1109_3186_gb300 import skymodel
from paper_1109_3186_gb300.chimg import ChimgPlan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K_DM = skymodel.K_DM
# relative error of every E entry above 1e-3 of its DM's largest value
REL_E_ABOVE_FLOOR = 1e-2
F0, BW = 1.4e9, 8e6


def _voltages(M, D, n_samp, dm, L, seed, l_dir, amp):
    y = skymodel.noise(M, n_samp, seed).astype(np.complex128)
    if amp:
        _, a0, a1 = ocpi.chirp_model(F0, BW, K_DM, dm)
        nw = ocpi.window_blocks(F0, BW, K_DM, dm, L)
        tc = (2 * L + nw * L / 2.0) / BW
        t = np.arange(n_samp) / BW
        for p in range(M):
            tau = p * D * l_dir / 299792458.0
            u = t - tc - tau
            y[p] += amp * np.exp(2j * math.pi * ((a0 - F0) * u + 0.5 * a1 * u * u)) \
                * np.exp(-2j * math.pi * F0 * tau)
    return y.astype(np.complex64)


CASES = {
    "8ant_natural": (8, 40.0, 1 << 14, [5.0, 20.0], 256, 16, 1, "natural", 31, 12, 0.5),
    "5ant_uniform_ragged_F0": (5, 80.0, 64 * 50 + 7, [2.0, 6.0], 64, 8, 0, "uniform", 32, 7, 0.0),
    "32ant_F2": (32, 20.0, 1 << 13, [3.0], 128, 64, 2, "natural", 33, 9, 0.3),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_grid_and_image_match_the_oracle(name):
    M, D, n, dms, L, Ns, F, w, seed, n_pix, amp = CASES[name]
    l_dirs = np.linspace(-0.01, 0.01, n_pix)
    y = _voltages(M, D, n, dms[-1], L, seed, l_dirs[n_pix // 3], amp)
    Yo = ochimg.integrate(ochimg.spatial_dft(ochimg.mix_grid(y, w), Ns), L)      # [Ns][n_dump]
    Eo = ochimg.image(Yo, M, D, l_dirs, F0, BW, K_DM, dms, L, Ns, F, w)
    with ChimgPlan(M, D, F0, BW, n, dms, L, l_dirs, Ns, F, weights=w, k_dm=K_DM) as plan:
        assert plan.n_dump == Yo.shape[1]
        assert list(plan.n_win) == [ocpi.window_blocks(F0, BW, K_DM, dm, L) for dm in dms]
        Y = np.empty((plan.n_dump, Ns), np.complex64)
        plan.grid(y, Y)
        assert np.abs(Y - Yo.T).max() <= 1e-5 * np.abs(Yo).max()
        E = np.empty((len(dms), plan.n_dump, n_pix), np.float32)
        plan.run(y, E)
        Ed = torch.empty(E.shape, dtype=torch.float32, device="cuda")
        plan.run(torch.from_numpy(y).cuda(), Ed)
        assert np.array_equal(E, Ed.cpu().numpy())
        for d in range(len(dms)):
            assert np.all(E[d][Eo[d] == 0] == 0)
            assert np.abs(E[d] - Eo[d]).max() <= 1e-4 * Eo[d].max(), d
            # element by element above a floor of 1e-3 of the DM's largest value
            big = Eo[d] > 1e-3 * Eo[d].max()
            rel = float((np.abs(E[d] - Eo[d])[big] / Eo[d][big]).max())
            print("chimg %s DM %d: max relative error of E above the floor %.3g" % (name, d, rel))
            assert rel <= REL_E_ABOVE_FLOOR, (d, rel)


# ------------------------------------------------ uniform rectangular arrays
from paper_1109_3186_gb300.chimg import Chimg2dPlan  # noqa: E402


def _voltages_2d(Mx, My, Dx, Dy, n_samp, dm, L, seed, lm, amp):
    """Noise plus one linear chirp (the oracle's trial model) from (l, m)."""
    y = skymodel.noise(Mx * My, n_samp, seed).astype(np.complex128)
    if amp:
        _, a0, a1 = ocpi.chirp_model(F0, BW, K_DM, dm)
        nw = ocpi.window_blocks(F0, BW, K_DM, dm, L)
        tc = (2 * L + nw * L / 2.0) / BW
        t = np.arange(n_samp) / BW
        for iy in range(My):
            for ix in range(Mx):
                tau = (ix * Dx * lm[0] + iy * Dy * lm[1]) / 299792458.0
                u = t - tc - tau
                y[iy * Mx + ix] += amp * np.exp(2j * math.pi * ((a0 - F0) * u + 0.5 * a1 * u * u)) \
                    * np.exp(-2j * math.pi * F0 * tau)
    return y.astype(np.complex64)


CASES_2D = {
    # Mx, My, Dx, Dy, n_samp, dms, L, (Nx, Ny), (Fx, Fy), weights, seed, n_side, amp
    "3x3_natural": (3, 3, 70.0, 50.0, 64 * 80, [8.0, 16.0], 64, (8, 8), (1, 1), "natural", 41, 3,
                    0.5),
    "4x2_uniform_ragged": (4, 2, 60.0, 90.0, 64 * 70 + 5, [6.0], 64, (8, 4), (2, 0), "uniform", 42,
                           3, 0.0),
    "2x4_natural_F0": (2, 4, 80.0, 40.0, 128 * 30, [10.0], 128, (4, 8), (0, 1), "natural", 43, 2,
                       0.4),
}


@pytest.mark.parametrize("name", sorted(CASES_2D))
def test_rectangular_grid_and_image_match_the_oracle(name):
    Mx, My, Dx, Dy, n, dms, L, (Nx, Ny), (Fx, Fy), w, seed, ns, amp = CASES_2D[name]
    ang = np.linspace(-0.004, 0.004, ns)
    pix = np.array([(a, b) for b in ang for a in ang])
    y = _voltages_2d(Mx, My, Dx, Dy, n, dms[-1], L, seed, pix[len(pix) // 2 - 1], amp)
    keys, _ = ochimg.spacings_2d(Mx, My)
    Xs = ochimg.spatial_dft_2d(ochimg.mix_grid_2d(y, Mx, My, w), Mx, My, Nx, Ny)
    nd = Xs.shape[2] // L
    Yo = Xs[:, :, :nd * L].reshape(Nx, Ny, nd, L).sum(axis=3)              # [Nx][Ny][n_dump]
    Eo = ochimg.search_2d(y, Mx, My, Dx, Dy, pix, F0, BW, K_DM, dms, L, Nx, Ny, (Fx, Fy), w)
    with Chimg2dPlan(Mx, My, Dx, Dy, F0, BW, n, dms, L, pix, (Nx, Ny), (Fx, Fy), weights=w,
                     k_dm=K_DM) as plan:
        assert plan.n_dump == nd and plan.n_spacing == len(keys)
        assert list(plan.n_win) == [ocpi.window_blocks(F0, BW, K_DM, dm, L) for dm in dms]
        Y = np.empty((nd, Nx, Ny), np.complex64)
        plan.grid(y, Y)
        assert np.abs(Y - Yo.transpose(2, 0, 1)).max() <= 1e-5 * np.abs(Yo).max()
        E = np.empty((len(dms), nd, len(pix)), np.float32)
        plan.run(y, E)
        Ed = torch.empty(E.shape, dtype=torch.float32, device="cuda")
        plan.run(torch.from_numpy(y).cuda(), Ed)
        assert np.array_equal(E, Ed.cpu().numpy())
    for d in range(len(dms)):
        assert np.all(E[d][Eo[d] == 0] == 0)
        assert np.abs(E[d] - Eo[d]).max() <= 1e-4 * Eo[d].max(), d
        big = Eo[d] > 1e-3 * Eo[d].max()
        rel = float((np.abs(E[d] - Eo[d])[big] / Eo[d][big]).max())
        print("chimg2d %s DM %d: max relative error of E above the floor %.3g" % (name, d, rel))
        assert rel <= REL_E_ABOVE_FLOOR, (d, rel)


def test_one_row_rectangular_plan_equals_the_linear_array_plan():
    M, D, n, dms, L, Ns, F = 6, 60.0, 64 * 60, [5.0, 12.0], 64, 16, 1
    l_dirs = np.linspace(-0.01, 0.01, 5)
    y = _voltages(M, D, n, dms[-1], L, 44, l_dirs[1], 0.4)
    E1 = np.empty((len(dms), n // L, len(l_dirs)), np.float32)
    E2 = np.empty_like(E1)
    with ChimgPlan(M, D, F0, BW, n, dms, L, l_dirs, Ns, F, k_dm=K_DM) as p1:
        p1.run(y, E1)
    pix = np.array([(l, 0.0) for l in l_dirs])
    with Chimg2dPlan(M, 1, D, 1.0, F0, BW, n, dms, L, pix, (Ns, 1), (F, 0), k_dm=K_DM) as p2:
        p2.run(y, E2)
    for d in range(len(dms)):
        assert np.abs(E1[d] - E2[d]).max() <= 2e-5 * E1[d].max()


def test_rectangular_plan_refuses_aliasing_grids():
    with pytest.raises(Exception) as ei:
        Chimg2dPlan(3, 3, 50.0, 50.0, F0, BW, 64 * 40, [8.0], 64, [(0.0, 0.0)], (4, 3), (0, 0))
    assert "n_spatial_x" in str(ei.value)
