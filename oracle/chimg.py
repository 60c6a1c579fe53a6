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
