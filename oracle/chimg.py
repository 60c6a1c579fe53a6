"""FP64 numpy oracle of the paper's own Chimageator pre-integrator on a
uniform linear array (Sec. 4.2, App. B.2): test infrastructure only.

Steps, for antennas p = 0..M-1 at positions p D along u (a uniform linear
array, Sec. 4.2):

1. Mixing (Eq. xpq_chimg): x_{p,p+l}[n] = y_p[n] y_{p+l}[n]^*.
2. Gridding: x'_l[n] = sum_{p=0}^{M-l-1} w_l x_{p,p+l}[n], l = 1..M-1 (the
   autocorrelations are not used); w_l = 1/(M - l) (the weighting the paper
   calls natural, whose weights sum to 1 per spacing) or w_l = 1.
3. Spatial DFT per sample (Sec. 4.2): X_k[n] = sum_{l=1}^{M-1}
   exp(-2 pi j k l / Ns) x'_l[n], k = 0..Ns-1 (x'_0 = 0; Ns >= M).
4. Integrate and dump (App. B.2.2): Y_k[m] = sum_{i<L} X_k[i + mL].
5. Trajectory sums (Eq. chimg_pth with the 2F widening of App. B.2.3): for a
   trial DM and direction, P = sum over the window's dumps m' of
   sum_{k = k0'(m') - F}^{k0'(m') + F} w_{k,m'} Y_k[m'], E = |P|^2 (Eq. eth).
6. The partial-sum recursion of App. B.2.1, in the paper's own model (below
   image()): trials of one trajectory gradient and intercept read their images
   from one cumulative sum along the line.

Readings (as for the Chirpolator pre-integrator: a baseband array and a
window-centred trial arrival):

* A trial DM is the linear chirp of Sec. 2.1 (rate fdot = a_1, centre a_0,
  sweep T); its window spans n_win = max(1, floor(B T / L + 1/2)) dumps and
  the chirp's temporal midpoint t_c is the window centre.
* Direction cosine l_dir along the array: tau_p = p D l_dir / c (Eq. tau3D).
  Pair (p, p+l) of a unit chirp then carries
      exp(2 pi j l tau (a_0 + fdot (t - t_c))) exp(pi j fdot tau^2 (p^2 - (p+l)^2)),
  a spatial tone of nu(t) = tau (a_0 + fdot (t - t_c)) cycles per spacing:
  the paper's trajectory k_0(n) = fdot tau Ns n / f_s (Eq. chimgf0) plus the
  carrier's constant offset Ns tau a_0 (bins taken modulo Ns).
* The filter of dump m' is the conjugate of the expected Y_k[m'] of a unit
  chirp from the trial direction (its exact sum over the dump's samples),
  divided by (M - 1) L, over the 2F+1 bins around rint(Ns nu(t_{m'})) (mod
  Ns), t_{m'} the dump's centre.  A perfect chirp gives
  P = sum_{m'} sum_k |Yhat_k[m']|^2 / ((M - 1) L) exactly.
"""

from __future__ import annotations

import math

import numpy as np

from . import cpi

C_LIGHT = 299792458.0


def mix_grid(y, weights: str = "natural") -> np.ndarray:
    """x'[l - 1][n] for l = 1..M-1 (steps 1 and 2)."""
    y = np.asarray(y, np.complex128)
    M = y.shape[0]
    out = np.zeros((M - 1, y.shape[1]), np.complex128)
    for l in range(1, M):
        w = 1.0 / (M - l) if weights == "natural" else 1.0
        for p in range(M - l):
            out[l - 1] += w * y[p] * np.conj(y[p + l])
    return out


def spatial_dft(xg, Ns: int) -> np.ndarray:
    """X[k][n] = sum_{l=1}^{M-1} exp(-2 pi j k l / Ns) x'_l[n] (step 3)."""
    L1 = xg.shape[0]
    basis = np.exp(-2j * math.pi * np.outer(np.arange(Ns), np.arange(1, L1 + 1)) / Ns)
    return basis @ xg


def integrate(X, L: int) -> np.ndarray:
    """Y[k][m] = sum_{i<L} X[k][i + mL], m < floor(n / L) (step 4)."""
    n_dump = X.shape[1] // L
    return X[:, :n_dump * L].reshape(X.shape[0], n_dump, L).sum(axis=2)


def expected_y(M, D, l_dir, f0, bw, k_dm, dm, L, Ns, m_rel, weights="natural"):
    """Expected Y[k] of a unit linear chirp from direction l_dir in the dump
    m_rel dumps after the window's first, window centred on the chirp."""
    _, a0, a1 = cpi.chirp_model(f0, bw, k_dm, dm)
    n_win = cpi.window_blocks(f0, bw, k_dm, dm, L)
    tau = D * l_dir / C_LIGHT
    t = (m_rel * L + np.arange(L) - n_win * L / 2.0) / bw            # t - t_c per sample
    xg = np.zeros((M - 1, L), np.complex128)
    for l in range(1, M):
        w = 1.0 / (M - l) if weights == "natural" else 1.0
        g = sum(np.exp(1j * math.pi * a1 * tau * tau * (p * p - (p + l) ** 2)) for p in range(M - l))
        xg[l - 1] = w * g * np.exp(2j * math.pi * l * tau * (a0 + a1 * t))
    return spatial_dft(xg, Ns).sum(axis=1)


def trajectory_bins(D, l_dir, f0, bw, k_dm, dm, L, Ns, m_rel):
    """rint(Ns nu) at the dump's centre, modulo Ns."""
    _, a0, a1 = cpi.chirp_model(f0, bw, k_dm, dm)
    n_win = cpi.window_blocks(f0, bw, k_dm, dm, L)
    tau = D * l_dir / C_LIGHT
    tm = (m_rel * L + (L - 1) / 2.0 - n_win * L / 2.0) / bw
    return int(np.rint(Ns * tau * (a0 + a1 * tm))) % Ns


def image(Y, M, D, l_dirs, f0, bw, k_dm, dms, L, Ns, F, weights="natural") -> np.ndarray:
    """E[d][m][pix] = |P|^2 for the window of n_win dumps ending at dump m
    (zero while m < n_win - 1), step 5."""
    n_dump = Y.shape[1]
    E = np.zeros((len(dms), n_dump, len(l_dirs)))
    for d, dm in enumerate(dms):
        n_win = cpi.window_blocks(f0, bw, k_dm, dm, L)
        for i, ld in enumerate(l_dirs):
            taps = []
            for r in range(n_win):
                yh = expected_y(M, D, ld, f0, bw, k_dm, dm, L, Ns, r, weights)
                kc = trajectory_bins(D, ld, f0, bw, k_dm, dm, L, Ns, r)
                ks = [(kc + j) % Ns for j in range(-F, F + 1)]
                taps.append((ks, np.conj(yh[ks]) / ((M - 1) * L)))
            for m in range(n_win - 1, n_dump):
                P = 0j
                for r, (ks, w) in enumerate(taps):
                    P += np.sum(w * Y[ks, m - n_win + 1 + r])
                E[d, m, i] = abs(P) ** 2
    return E


def search(y, D, l_dirs, f0, bw, k_dm, dms, L, Ns, F, weights="natural"):
    """E[d][m][pix] from raw voltages y [M][n] of a uniform linear array."""
    M = np.asarray(y).shape[0]
    Y = integrate(spatial_dft(mix_grid(y, weights), Ns), L)
    return image(Y, M, D, l_dirs, f0, bw, k_dm, dms, L, Ns, F, weights)


# ------------------------------------- App. B.2.1: shared partial sums
# The paper's own model of Sec. 4.2 (Eq. chimg_xpq with its tau^2 term dropped,
# natural weights summing to 1 per spacing, a baseband chirp that sweeps 0..B
# from the window start) puts the spatial tone nu(t) = fdot tau t cycles per
# spacing on the grid, t counted from the window start: the trajectory
# k_0(n) = Ns fdot tau n / f_s of Eq. chimgf0 passes through k = 0 at the start
# with a gradient set by rate = fdot tau alone.  With fdot = B / T a trial of
# sweep T from direction tau has rate tau B / T, and the trials of one rate --
# one gradient (Eq. chimg_grad), one intercept -- lie on one line: each one's
# image over a window starting at dump s is a prefix of one cumulative sum
# along the line from s (App. B.2.1).

def paper_expected_y(M, rate, bw, L, Ns, m_rel) -> np.ndarray:
    """Expected Y[k] of a unit chirp in the paper's model, dump m_rel of the
    window (samples t = (m_rel L + i) / B from the window start)."""
    t = (m_rel * L + np.arange(L)) / bw
    xg = np.exp(2j * math.pi * np.outer(np.arange(1, M), rate * t))
    return spatial_dft(xg, Ns).sum(axis=1)


def paper_taps(M, rate, bw, L, Ns, F, n_win):
    """Per dump r < n_win of the window: the 2F+1 bins around rint(Ns nu) at
    the dump's centre (mod Ns) and the conjugate expected Y there over
    (M - 1) L, as in image()."""
    taps = []
    for r in range(n_win):
        yh = paper_expected_y(M, rate, bw, L, Ns, r)
        kc = int(np.rint(Ns * rate * (r * L + (L - 1) / 2.0) / bw)) % Ns
        ks = [(kc + j) % Ns for j in range(-F, F + 1)]
        taps.append((ks, np.conj(yh[ks]) / ((M - 1) * L)))
    return taps


def prefix_sums(Y, taps, start) -> np.ndarray:
    """S[r] = sum_{r' <= r} sum_j w Y[k][start + r'] along the taps (the
    cumulative trajectory sum of App. B.2.1), for r < len(taps)."""
    S = np.zeros(len(taps), np.complex128)
    acc = 0j
    for r, (ks, w) in enumerate(taps):
        acc += np.sum(w * Y[ks, start + r])
        S[r] = acc
    return S


def paper_image_direct(Y, M, rate, n_wins, bw, L, Ns, F) -> np.ndarray:
    """E[i][m] of the trials with n_wins[i] dumps on the line `rate`, each from
    its own taps (Eq. chimg_pth), for windows ending at dump m (zero while
    m < n_win - 1)."""
    n_dump = Y.shape[1]
    E = np.zeros((len(n_wins), n_dump))
    for i, nw in enumerate(n_wins):
        taps = paper_taps(M, rate, bw, L, Ns, F, nw)
        for m in range(nw - 1, n_dump):
            P = 0j
            for r, (ks, w) in enumerate(taps):
                P += np.sum(w * Y[ks, m - nw + 1 + r])
            E[i, m] = abs(P) ** 2
    return E


def paper_image_shared(Y, M, rate, n_wins, bw, L, Ns, F) -> np.ndarray:
    """The same images by the recursion of App. B.2.1: one cumulative sum
    along the line per window start, with the longest trial's taps, read at
    each trial's length."""
    n_dump = Y.shape[1]
    n_max = max(n_wins)
    taps = paper_taps(M, rate, bw, L, Ns, F, n_max)
    E = np.zeros((len(n_wins), n_dump))
    for s in range(n_dump):
        S = prefix_sums(Y, taps[:min(n_max, n_dump - s)], s)
        for i, nw in enumerate(n_wins):
            if nw <= len(S):
                E[i, s + nw - 1] = abs(S[nw - 1]) ** 2
    return E


# ------------------------------------------------ uniform rectangular array
# Antenna a = iy * Mx + ix at (ix Dx, iy Dy, 0).  Spacings (lx, ly) of the
# half plane ly > 0, or ly = 0 and lx > 0, each gridded as the weighted sum of
# its pairs (p, q = p + (lx, ly)); the spatial DFT is 2-D over that grid:
#   X[kx][ky][n] = sum_{lx,ly} exp(-2 pi j (kx lx / Nx + ky ly / Ny)) x'_{lx,ly}[n].
# A unit chirp from (l, m) puts the tone nu = (Dx l, Dy m)(a_0 + fdot (t - t_c))/c
# cycles per spacing on the grid; the trajectory sums take (2Fx+1)(2Fy+1) bins
# per dump around (rint(Nx nu_x), rint(Ny nu_y)) (mod Nx, Ny) with the conjugate
# expected Y divided by (number of spacings) L.  With My = 1, Ny = 1 and
# Fy = 0 every step is the uniform linear array's.

def spacings_2d(Mx: int, My: int):
    """Half-plane spacings (lx, ly) and, for each, its pairs (p, q)."""
    out = {}
    for iy in range(My):
        for ix in range(Mx):
            for jy in range(My):
                for jx in range(Mx):
                    lx, ly = jx - ix, jy - iy
                    if ly > 0 or (ly == 0 and lx > 0):
                        out.setdefault((lx, ly), []).append((iy * Mx + ix, jy * Mx + jx))
    keys = sorted(out, key=lambda s: (s[1], s[0]))
    return keys, [out[k] for k in keys]


def mix_grid_2d(y, Mx: int, My: int, weights: str = "natural"):
    """x'[s][n] for the half-plane spacings s (steps 1 and 2)."""
    y = np.asarray(y, np.complex128)
    keys, prs = spacings_2d(Mx, My)
    out = np.zeros((len(keys), y.shape[1]), np.complex128)
    for s, pl in enumerate(prs):
        w = 1.0 / len(pl) if weights == "natural" else 1.0
        for p, q in pl:
            out[s] += w * y[p] * np.conj(y[q])
    return out


def check_grid_2d(Mx: int, My: int, Nx: int, Ny: int):
    """The half-plane spacings run lx = -(Mx-1)..(Mx-1) and ly = 0..(My-1): a
    grid with Nx < 2 Mx - 1 or Ny < My would fold distinct spacings onto one
    DFT bin (aliasing), so it is refused.  One row (My = 1) has lx = 1..Mx-1
    only and needs Nx >= Mx (the linear array's rule) and Ny >= 1."""
    nx_min = Mx if My == 1 else 2 * Mx - 1
    if Nx < nx_min or Ny < My or Ny < 1:
        raise ValueError("spatial grid %dx%d aliases the spacings of a %dx%d array "
                         "(need Nx >= %d, Ny >= %d)" % (Nx, Ny, Mx, My, nx_min, My))


def spatial_dft_2d(xg, Mx: int, My: int, Nx: int, Ny: int):
    """X[kx][ky][n] over the half-plane grid (step 3)."""
    check_grid_2d(Mx, My, Nx, Ny)
    keys, _ = spacings_2d(Mx, My)
    kx = np.arange(Nx)[:, None, None]
    ky = np.arange(Ny)[None, :, None]
    lx = np.array([k[0] for k in keys])[None, None, :]
    ly = np.array([k[1] for k in keys])[None, None, :]
    basis = np.exp(-2j * math.pi * (kx * lx / Nx + ky * ly / Ny))          # [Nx][Ny][S]
    return np.einsum("abs,sn->abn", basis, xg)


def expected_y_2d(Mx, My, Dx, Dy, l, m, f0, bw, k_dm, dm, L, Nx, Ny, m_rel, weights="natural"):
    """Expected Y[kx][ky] of a unit linear chirp from (l, m) in dump m_rel of the window."""
    _, a0, a1 = cpi.chirp_model(f0, bw, k_dm, dm)
    n_win = cpi.window_blocks(f0, bw, k_dm, dm, L)
    t = (m_rel * L + np.arange(L) - n_win * L / 2.0) / bw
    pos = [(ix * Dx, iy * Dy) for iy in range(My) for ix in range(Mx)]
    tau = np.array([(px * l + py * m) / C_LIGHT for px, py in pos])
    keys, prs = spacings_2d(Mx, My)
    xg = np.zeros((len(keys), L), np.complex128)
    for s, pl in enumerate(prs):
        w = 1.0 / len(pl) if weights == "natural" else 1.0
        for p, q in pl:
            dt = tau[p] - tau[q]
            xg[s] += w * np.exp(-2j * math.pi * dt * (a0 + a1 * t)) \
                * np.exp(1j * math.pi * a1 * (tau[p] ** 2 - tau[q] ** 2))
    return spatial_dft_2d(xg, Mx, My, Nx, Ny).sum(axis=2)


def trajectory_bins_2d(Dx, Dy, l, m, f0, bw, k_dm, dm, L, Nx, Ny, m_rel):
    _, a0, a1 = cpi.chirp_model(f0, bw, k_dm, dm)
    n_win = cpi.window_blocks(f0, bw, k_dm, dm, L)
    tm = (m_rel * L + (L - 1) / 2.0 - n_win * L / 2.0) / bw
    fr = a0 + a1 * tm
    return (int(np.rint(Nx * Dx * l * fr / C_LIGHT)) % Nx, int(np.rint(Ny * Dy * m * fr / C_LIGHT)) % Ny)


def search_2d(y, Mx, My, Dx, Dy, pix_lm, f0, bw, k_dm, dms, L, Nx, Ny, F, weights="natural"):
    """E[d][m][pix] for a uniform rectangular array (steps 1-5); F is the
    half width (Fx, Fy) of the bin neighbourhood, or one value for both."""
    Fx, Fy = (F, F) if np.isscalar(F) else F
    check_grid_2d(Mx, My, Nx, Ny)
    keys, _ = spacings_2d(Mx, My)
    Xs = spatial_dft_2d(mix_grid_2d(y, Mx, My, weights), Mx, My, Nx, Ny)
    n_dump = Xs.shape[2] // L
    Y = Xs[:, :, :n_dump * L].reshape(Nx, Ny, n_dump, L).sum(axis=3)
    E = np.zeros((len(dms), n_dump, len(pix_lm)))
    for d, dm in enumerate(dms):
        n_win = cpi.window_blocks(f0, bw, k_dm, dm, L)
        for i, (l, m) in enumerate(np.asarray(pix_lm, np.float64)):
            taps = []
            for r in range(n_win):
                yh = expected_y_2d(Mx, My, Dx, Dy, l, m, f0, bw, k_dm, dm, L, Nx, Ny, r, weights)
                cx, cy = trajectory_bins_2d(Dx, Dy, l, m, f0, bw, k_dm, dm, L, Nx, Ny, r)
                kk = [((cx + jx) % Nx, (cy + jy) % Ny) for jx in range(-Fx, Fx + 1) for jy in range(-Fy, Fy + 1)]
                taps.append((kk, np.array([np.conj(yh[a, b]) for a, b in kk]) / (len(keys) * L)))
            for mm in range(n_win - 1, n_dump):
                P = 0j
                for r, (kk, w) in enumerate(taps):
                    col = mm - n_win + 1 + r
                    P += np.sum(w * np.array([Y[a, b, col] for a, b in kk]))
                E[d, mm, i] = abs(P) ** 2
    return E
