"""Pins of the Chimageator pre-integrator oracle (oracle/chimg.py) against the
physics and closed forms: gridded products of a linear chirp on a uniform
linear array (Sec. 4.2), the spatial DFT's Dirichlet-type response, the
trajectory of the peak bin (Eq. chimgf0), integrate-and-dump (App. B.2.2),
the exact image of a perfect chirp and its peak at the true direction and
DM (Eqs. chimg_pth, eth), and planted mistakes."""
import math

import numpy as np
import pytest

from oracle import chimg, cpi

K_DM = 4.148808e15
C = 299792458.0


def _chirp_ula(M, D, l_dir, f0, bw, dm, L, m_first, n_samp):
    """Baseband voltages of a unit linear chirp (rate a1, centre a0, midpoint
    at the centre of the window whose first dump is m_first) from direction
    l_dir on antennas p D: y_p(t) = s(t - tau_p) exp(-2 pi j f0 tau_p)."""
    _, a0, a1 = cpi.chirp_model(f0, bw, K_DM, dm)
    n_win = cpi.window_blocks(f0, bw, K_DM, dm, L)
    tc = (m_first * L + n_win * L / 2.0) / bw
    t = np.arange(n_samp) / bw
    y = np.empty((M, n_samp), np.complex128)
    for p in range(M):
        tau = p * D * l_dir / C
        u = t - tc - tau
        y[p] = np.exp(2j * math.pi * ((a0 - f0) * u + 0.5 * a1 * u * u)) * np.exp(-2j * math.pi * f0 * tau)
    return y, n_win, tc


def test_gridded_chirp_is_a_spatial_tone():
    M, D, l_dir, f0, bw, dm, L = 6, 40.0, 0.01, 1.4e9, 8e6, 20.0, 64
    y, n_win, tc = _chirp_ula(M, D, l_dir, f0, bw, dm, L, 0, 8 * L)
    _, a0, a1 = cpi.chirp_model(f0, bw, K_DM, dm)
    tau = D * l_dir / C
    t = np.arange(y.shape[1]) / bw - tc
    xg = chimg.mix_grid(y)
    for l in range(1, M):
        g = np.mean([np.exp(-1j * math.pi * a1 * tau * tau * l * (2 * p + l)) for p in range(M - l)])
        want = g * np.exp(2j * math.pi * l * tau * (a0 + a1 * t))
        assert np.abs(xg[l - 1] - want).max() < 1e-9
    xu = chimg.mix_grid(y, weights="uniform")
    assert np.abs(xu[0] - (M - 1) * xg[0]).max() < 1e-9


def test_spatial_dft_of_a_tone_is_the_shifted_dirichlet_form():
    M, Ns = 7, 16
    for nu in (0.13, -0.31, 2.6):
        xg = np.exp(2j * math.pi * np.arange(1, M)[:, None] * nu) * np.ones((1, 3))
        X = chimg.spatial_dft(xg, Ns)[:, 0]
        for k in range(Ns):
            x = nu - k / Ns
            want = np.exp(1j * math.pi * M * x) * math.sin(math.pi * (M - 1) * x) / math.sin(math.pi * x)
            assert abs(X[k] - want) < 1e-9


def test_peak_bin_moves_along_the_trajectory():
    # Eq. chimgf0 without a carrier: x'_l[n] = exp(2 pi j fdot tau l n / f_s) peaks at k0 = fdot tau Ns n / f_s
    M, Ns, fs = 8, 64, 1e6
    fdot, tau = 2e9, 3e-9
    n = np.arange(0, 4000, 500)
    xg = np.exp(2j * math.pi * np.arange(1, M)[:, None] * fdot * tau * n[None, :] / fs)
    X = chimg.spatial_dft(xg, Ns)
    for c, nn in enumerate(n):
        k0 = (fdot * tau * Ns * nn / fs) % Ns
        got = int(np.argmax(np.abs(X[:, c])))
        assert min(abs(got - k0), Ns - abs(got - k0)) <= 0.5


def test_integrate_and_dump():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((5, 103)) + 1j * rng.standard_normal((5, 103))
    Y = chimg.integrate(X, 10)
    assert Y.shape == (5, 10)
    for m in (0, 4, 9):
        assert np.abs(Y[:, m] - X[:, m * 10:(m + 1) * 10].sum(axis=1)).max() < 1e-12


def _perfect_case(mix_fn=None):
    M, D, f0, bw, L, Ns, F = 6, 60.0, 1.4e9, 8e6, 64, 16, 1
    dms = [8.0, 16.0, 32.0]
    l_dirs = [-0.004, 0.0, 0.003, 0.006]
    true_d, true_i = 1, 2
    n_win = cpi.window_blocks(f0, bw, K_DM, dms[true_d], L)
    m_first = 3
    y, _, _ = _chirp_ula(M, D, l_dirs[true_i], f0, bw, dms[true_d], L, m_first, (m_first + n_win + 3) * L)
    if mix_fn is not None:
        xg = mix_fn(y)
        Y = chimg.integrate(chimg.spatial_dft(xg, Ns), L)
        E = chimg.image(Y, M, D, l_dirs, f0, bw, K_DM, dms, L, Ns, F)
    else:
        E = chimg.search(y, D, l_dirs, f0, bw, K_DM, dms, L, Ns, F)
    m_end = m_first + n_win - 1
    P = 0.0
    for r in range(n_win):
        yh = chimg.expected_y(M, D, l_dirs[true_i], f0, bw, K_DM, dms[true_d], L, Ns, r)
        kc = chimg.trajectory_bins(D, l_dirs[true_i], f0, bw, K_DM, dms[true_d], L, Ns, r)
        ks = [(kc + j) % Ns for j in range(-F, F + 1)]
        P += float(np.sum(np.abs(yh[ks]) ** 2)) / ((M - 1) * L)
    return E, true_d, true_i, m_end, P, n_win


def test_image_of_a_perfect_chirp_is_exact_and_peaks_at_its_direction():
    E, d, i, m_end, P, n_win = _perfect_case()
    assert abs(E[d, m_end, i] - P * P) < 1e-9 * P * P
    assert int(np.argmax(E[d, m_end])) == i
    assert np.all(E[d, :n_win - 1] == 0)


def test_planted_mistakes_fail_the_perfect_chirp_pin():
    def mix_conj(y):  # y_q y_p^* instead of y_p y_q^*
        return np.conj(chimg.mix_grid(y))

    def mix_shift(y):  # spacing off by one
        g = chimg.mix_grid(y)
        return np.vstack([g[1:], np.zeros_like(g[:1])])

    for bad in (mix_conj, mix_shift):
        E, d, i, m_end, P, _ = _perfect_case(bad)
        assert abs(E[d, m_end, i] - P * P) > 1e-3 * P * P


@pytest.mark.parametrize("Ns", [8, 12])
def test_spatial_dft_is_linear(Ns):
    rng = np.random.default_rng(Ns)
    a = rng.standard_normal((5, 4)) + 1j * rng.standard_normal((5, 4))
    b = rng.standard_normal((5, 4)) + 1j * rng.standard_normal((5, 4))
    assert np.abs(chimg.spatial_dft(2 * a - 1j * b, Ns) - (2 * chimg.spatial_dft(a, Ns) - 1j * chimg.spatial_dft(b, Ns))).max() < 1e-12


def test_rectangular_array_with_one_row_is_the_linear_array():
    M, D, f0, bw, L, Ns, F = 6, 60.0, 1.4e9, 8e6, 64, 16, 1
    dms = [8.0, 16.0]
    l_dirs = [-0.004, 0.003]
    y, _, _ = _chirp_ula(M, D, 0.003, f0, bw, 16.0, L, 3, 30 * L)
    y = y + 0.3 * (np.random.default_rng(1).standard_normal(y.shape))
    E1 = chimg.search(y, D, l_dirs, f0, bw, K_DM, dms, L, Ns, F)
    E2 = chimg.search_2d(y, M, 1, D, 1.0, [(l, 0.0) for l in l_dirs], f0, bw, K_DM, dms, L, Ns, 1,
                         (F, 0))
    assert np.abs(E1 - E2).max() <= 1e-10 * E1.max()


def _chirp_ura(Mx, My, Dx, Dy, l, m, f0, bw, dm, L, m_first, n_samp):
    _, a0, a1 = cpi.chirp_model(f0, bw, K_DM, dm)
    n_win = cpi.window_blocks(f0, bw, K_DM, dm, L)
    tc = (m_first * L + n_win * L / 2.0) / bw
    t = np.arange(n_samp) / bw
    y = np.empty((Mx * My, n_samp), np.complex128)
    for iy in range(My):
        for ix in range(Mx):
            tau = (ix * Dx * l + iy * Dy * m) / C
            u = t - tc - tau
            y[iy * Mx + ix] = np.exp(2j * math.pi * ((a0 - f0) * u + 0.5 * a1 * u * u)) \
                * np.exp(-2j * math.pi * f0 * tau)
    return y, n_win


def test_rectangular_array_image_of_a_perfect_chirp_is_exact_and_peaks_at_its_pixel():
    Mx, My, Dx, Dy, f0, bw, L, Nx, Ny, F, dm = 3, 3, 70.0, 50.0, 1.4e9, 8e6, 64, 8, 8, 1, 16.0
    ang = np.linspace(-0.004, 0.004, 3)
    pix = [(a, b) for b in ang for a in ang]
    true = 5
    n_win = cpi.window_blocks(f0, bw, K_DM, dm, L)
    y, _ = _chirp_ura(Mx, My, Dx, Dy, *pix[true], f0, bw, dm, L, 2, (n_win + 4) * L)
    E = chimg.search_2d(y, Mx, My, Dx, Dy, pix, f0, bw, K_DM, [dm], L, Nx, Ny, F)
    keys, _ = chimg.spacings_2d(Mx, My)
    P = 0.0
    for r in range(n_win):
        yh = chimg.expected_y_2d(Mx, My, Dx, Dy, *pix[true], f0, bw, K_DM, dm, L, Nx, Ny, r)
        cx, cy = chimg.trajectory_bins_2d(Dx, Dy, *pix[true], f0, bw, K_DM, dm, L, Nx, Ny, r)
        for jx in range(-F, F + 1):
            for jy in range(-F, F + 1):
                P += abs(yh[(cx + jx) % Nx, (cy + jy) % Ny]) ** 2 / (len(keys) * L)
    m_end = 2 + n_win - 1
    assert abs(E[0, m_end, true] - P * P) < 1e-9 * P * P
    assert int(np.argmax(E[0, m_end])) == true


def test_rectangular_grids_that_alias_spacings_are_refused():
    """Spacings lx = -(Mx-1)..(Mx-1), ly = 0..(My-1) need Nx >= 2 Mx - 1 and
    Ny >= My to land on distinct bins; one row needs only Nx >= Mx."""
    y = np.ones((9, 64), np.complex128)
    xg = chimg.mix_grid_2d(y, 3, 3)
    chimg.spatial_dft_2d(xg, 3, 3, 5, 3)
    for nx, ny in ((4, 3), (5, 2)):
        with pytest.raises(ValueError):
            chimg.spatial_dft_2d(xg, 3, 3, nx, ny)
    with pytest.raises(ValueError):
        chimg.search_2d(y, 3, 3, 50.0, 50.0, [(0.0, 0.0)], 1.4e9, 8e6, K_DM, [8.0], 16, 4, 3, 0)
    chimg.spatial_dft_2d(chimg.mix_grid_2d(y[:4], 4, 1), 4, 1, 4, 1)
    with pytest.raises(ValueError):
        chimg.spatial_dft_2d(chimg.mix_grid_2d(y[:4], 4, 1), 4, 1, 3, 1)
