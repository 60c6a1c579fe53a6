"""FP64 numpy oracle of the paper's own Chirpolator pre-integrator (test
infrastructure only: tests, the smoke check and the benchmark's CPU leg use
it; the product never does).

The Chirpolator (Sec. 3) searches the RAW (not dedispersed) voltages:

1. Mixing (Eq. xpq): x_pq[n] = y_p[n] y_q[n]^*, for every pair p < q (the
   autocorrelations are not used, Eq. pth sums q > p).  A dispersed pulse,
   modelled as a linear chirp of rate fdot (Sec. 2.1: fdot = a_1), becomes a
   tone of frequency -fdot (tau_p - tau_q) on pair pq.
2. Block-based sliding DFT (Sec. A.3.2): partial DFTs over blocks of L
   samples, with the phase measured from sample 0,
       V_k[m] = sum_{n<L} exp(-2 pi j (n + mL) k / N) x[n + mL],
   and the DFT over the N = n_win L samples ending with block m by the moving
   sum of Eq. block_cic:  S_k[m] = S_k[m-1] + V_k[m] - V_k[m - n_win].
   One trial DM fixes N: the sweep of a pulse across the band takes
   T = k DM ((f0 - B/2)^-2 - (f0 + B/2)^-2) (Eq. dmdelay), so N ~ B T.
3. Imaging (Eqs. pth, eth, and the 2F+1-bin matched filter of Sec. 3.4):
   P(l, m) = sum_{p<q} sum_{k = k0' - F}^{k0' + F} w_pq,k X_pq,k,
   E = |P|^2, with X the DFT in the window's own time (sample 0 = the
   window's first sample), k0' = rint(kappa) and w the conjugate of the
   response expected from a linear chirp out of direction (l, m).

Readings (the paper's derivation puts the window start at the chirp's zero
frequency and leaves out the carrier; a baseband array needs both):

* Linear chirp: rate fdot = a_1 and centre frequency a_0 of the Taylor
  expansion about the sweep's temporal midpoint (Sec. 2.1, Eq. freqvst2).
* Window: n_win = max(1, floor(B T / L + 1/2)) blocks; the chirp is assumed
  to sweep across the window with its temporal midpoint at the window centre.
* Expected response of pair pq to a unit linear chirp from direction (l, m),
  baseband voltages y_a(t) = s(t - tau_a) exp(-2 pi j f0 tau_a), tau from
  Eq. tau3D:  X_k = phi_pq exp(-pi j kappa) exp(-pi j (k - kappa)(N-1)/N)
  D_N(k - kappa), where kappa = -fdot (tau_p - tau_q) N / B (Eq. f0Bt,
  k_0 = fdot tau N / f_s, with the sign of fdot kept),
  phi_pq = exp(pi j fdot (tau_p^2 - tau_q^2) - 2 pi j a_0 (tau_p - tau_q)),
  and D_N the Dirichlet kernel of Eq. dn.  For the two-antenna case of
  Sec. 3.2 (tau_p = 0) phi_pq reduces to the first factor of Eq. phipq1.
* Matched filter: w_pq,k = conj(X_k / D_N(k - kappa)) D_N(k - kappa) / N, i.e.
  the conjugate expected phase weighted by the expected amplitude normalised
  to 1 at the peak (the D_N argument of Sec. 3.4 read as the bin's distance
  from the tone).  A perfect chirp of unit amplitude from the pixel's
  direction then gives P = sum_pq sum_k D_N(k - kappa)^2 / N exactly.
* Bins: every pair computes k in [-K, K]; pair pq needs only
  |k| <= K_pq = max over DMs and pixels of |rint(kappa)| + F (Sec. A.3.1).
* Outputs: block m < floor(n_samp / L); windows with m < n_win - 1 are
  incomplete and read as zero.

Written for checking by eye: explicit loops over pairs, DMs and blocks; a
matrix product stands for the sum over the L samples of a block.
"""

from __future__ import annotations

import math

import numpy as np

C_LIGHT = 299792458.0


# ----------------------------------------------------------------- model
def chirp_model(f0: float, bw: float, k_dm: float, dm: float):
    """(T, a0, a1): sweep time across the band (Eq. dmdelay), and the
    constant and linear Taylor coefficients of the instantaneous frequency
    about the sweep's temporal midpoint (Sec. 2.1, Eq. freqvst2)."""
    if dm <= 0.0:
        raise ValueError("the linear-chirp model needs DM > 0")
    nu_lo, nu_hi = f0 - 0.5 * bw, f0 + 0.5 * bw
    T = k_dm * dm * (nu_lo ** -2 - nu_hi ** -2)
    alpha = 0.5 * (nu_lo ** -2 + nu_hi ** -2)
    a0 = alpha ** -0.5
    a1 = -0.5 * alpha ** -1.5 / (k_dm * dm)
    return T, a0, a1


def window_blocks(f0, bw, k_dm, dm, blk_len) -> int:
    """n_win: blocks of L samples in the DFT window of a trial DM."""
    T, _, _ = chirp_model(f0, bw, k_dm, dm)
    return max(1, int(math.floor(bw * T / blk_len + 0.5)))


def pairs(n_ant: int):
    """Antenna pairs p < q in the order (0,1), (0,2), ..., (M-2, M-1)."""
    return [(p, q) for p in range(n_ant) for q in range(p + 1, n_ant)]


def delays(xyz, pix_lm) -> np.ndarray:
    """tau[pix][a] in seconds (Eq. tau3D)."""
    xyz = np.asarray(xyz, np.float64)
    out = np.empty((len(pix_lm), xyz.shape[0]))
    for i, (l, m) in enumerate(np.asarray(pix_lm, np.float64)):
        n = math.sqrt(max(0.0, 1.0 - l * l - m * m))
        out[i] = (xyz[:, 0] * l + xyz[:, 1] * m + xyz[:, 2] * (n - 1.0)) / C_LIGHT
    return out


def dirichlet(x, N: int):
    """D_N(x) of Eq. dn: N at x = 0, sin(pi x) / sin(pi x / N) elsewhere."""
    x = np.asarray(x, np.float64)
    out = np.full(x.shape, float(N))
    nz = np.abs(x) > 1e-12
    out[nz] = np.sin(math.pi * x[nz]) / np.sin(math.pi * x[nz] / N)
    return out


def kappa(tau_p, tau_q, fdot, n_fft, bw):
    """Tone of pair pq in DFT bins of an N-sample window (Eq. f0Bt)."""
    return -fdot * (tau_p - tau_q) * n_fft / bw


# ----------------------------------------------------------------- steps
def mix(y) -> np.ndarray:
    """x[pair][n] = y_p[n] conj(y_q[n]) (Eq. xpq)."""
    y = np.asarray(y, np.complex128)
    return np.stack([y[p] * np.conj(y[q]) for p, q in pairs(y.shape[0])])


def partial_dft(xpq, blk_len: int, n_fft: int, K: int) -> np.ndarray:
    """V[k + K][m][pair] = sum_{n<L} exp(-2 pi j (n + mL) k / N) x[pair][n + mL]
    for k in [-K, K], m < floor(n / L) (Sec. A.3.2)."""
    n_pair, n = xpq.shape
    n_blk = n // blk_len
    ks = np.arange(-K, K + 1)
    V = np.empty((2 * K + 1, n_blk, n_pair), np.complex128)
    for m in range(n_blk):
        idx = np.arange(blk_len) + m * blk_len
        basis = np.exp(-2j * math.pi * np.outer(ks, idx) / n_fft)     # [bins][L]
        V[:, m, :] = basis @ xpq[:, idx].T
    return V


def cic(V, n_win: int) -> np.ndarray:
    """S[k][m] = S[k][m-1] + V[k][m] - V[k][m - n_win] (Eq. block_cic), S[-1] = 0,
    V[m < 0] = 0."""
    S = np.zeros_like(V)
    run = np.zeros(V.shape[0:1] + V.shape[2:], V.dtype)
    for m in range(V.shape[1]):
        run = run + V[:, m]
        if m - n_win >= 0:
            run = run - V[:, m - n_win]
        S[:, m] = run
    return S


def window_local(S, n_win: int, K: int) -> np.ndarray:
    """X[k][m] = exp(2 pi j n0 k / N) S[k][m], n0 = (m + 1 - n_win) L the window's
    first sample, N = n_win L; zero for incomplete windows."""
    X = np.zeros_like(S)
    ks = np.arange(-K, K + 1)
    for m in range(n_win - 1, S.shape[1]):
        X[:, m] = np.exp(2j * math.pi * (m + 1 - n_win) * ks / n_win)[:, None] * S[:, m]
    return X


def image_weights(xyz, pix_lm, f0, bw, k_dm, dm, blk_len, F):
    """(k0p[pix][pair], W[pix][pair][2F+1]): first bin k0' - F and the matched
    filter over bins k0' - F .. k0' + F (Sec. 3.4 with the readings above)."""
    _, a0, a1 = chirp_model(f0, bw, k_dm, dm)
    n_win = window_blocks(f0, bw, k_dm, dm, blk_len)
    N = n_win * blk_len
    tau = delays(xyz, pix_lm)
    pl = pairs(np.asarray(xyz).shape[0])
    k0p = np.empty((len(pix_lm), len(pl)), np.int64)
    W = np.empty((len(pix_lm), len(pl), 2 * F + 1), np.complex128)
    for i in range(len(pix_lm)):
        for c, (p, q) in enumerate(pl):
            kap = kappa(tau[i, p], tau[i, q], a1, N, bw)
            phi = np.exp(1j * math.pi * a1 * (tau[i, p] ** 2 - tau[i, q] ** 2)
                         - 2j * math.pi * a0 * (tau[i, p] - tau[i, q]))
            kc = int(np.rint(kap))
            k = np.arange(kc - F, kc + F + 1)
            x = k - kap
            phase = phi * np.exp(-1j * math.pi * kap) * np.exp(-1j * math.pi * x * (N - 1) / N)
            W[i, c] = np.conj(phase) * dirichlet(x, N) / N
            k0p[i, c] = kc - F
    return k0p, W


def image(X, k0p, W, K: int) -> np.ndarray:
    """E[m][pix] = |sum_pair sum_j W[pix][pair][j] X[k0p + j + K][m][pair]|^2 (Eqs. pth, eth)."""
    n_pix, n_pair, nj = W.shape
    E = np.empty((X.shape[1], n_pix))
    for i in range(n_pix):
        P = np.zeros(X.shape[1], np.complex128)
        for c in range(n_pair):
            for j in range(nj):
                P += W[i, c, j] * X[k0p[i, c] + j + K, :, c]
        E[:, i] = np.abs(P) ** 2
    return E


def pair_bins(xyz, pix_lm, f0, bw, k_dm, dms, blk_len, F) -> np.ndarray:
    """K_pq = max over DMs and pixels of |rint(kappa)| + F (Sec. A.3.1)."""
    tau = delays(xyz, pix_lm)
    pl = pairs(np.asarray(xyz).shape[0])
    out = np.zeros(len(pl), np.int64)
    for dm in dms:
        _, _, a1 = chirp_model(f0, bw, k_dm, dm)
        N = window_blocks(f0, bw, k_dm, dm, blk_len) * blk_len
        for c, (p, q) in enumerate(pl):
            kap = kappa(tau[:, p], tau[:, q], a1, N, bw)
            out[c] = max(out[c], int(np.max(np.abs(np.rint(kap)))) + F)
    return out


def search(y, xyz, pix_lm, f0, bw, k_dm, dms, blk_len, F, K=None, keep=False):
    """E[d][m][pix] for every trial DM (and V, X per DM when keep)."""
    if K is None:
        K = int(pair_bins(xyz, pix_lm, f0, bw, k_dm, dms, blk_len, F).max())
    xpq = mix(y)
    n_blk = xpq.shape[1] // blk_len
    E = np.zeros((len(dms), n_blk, len(pix_lm)))
    kept = []
    for d, dm in enumerate(dms):
        n_win = window_blocks(f0, bw, k_dm, dm, blk_len)
        V = partial_dft(xpq, blk_len, n_win * blk_len, K)
        X = window_local(cic(V, n_win), n_win, K)
        k0p, W = image_weights(xyz, pix_lm, f0, bw, k_dm, dm, blk_len, F)
        if np.any(k0p < -K) or np.any(k0p + 2 * F > K):
            raise ValueError("K too small for the pixels' bins")
        E[d] = image(X, k0p, W, K)
        if keep:
            kept.append((V, X))
    return (E, kept, K) if keep else E


# ------------------------------------------------- planning quantities
def gauss_sum(a: float, L: int) -> complex:
    """G(a, L) = sum_{n<L} exp(2 pi j a n^2) (Eq. gaussum)."""
    n = np.arange(L, dtype=np.float64)
    return complex(np.sum(np.exp(2j * math.pi * a * n * n)))


def delta_mix(f0, bw, k_dm, dm, tau):
    """Smearing of the mixed tone at the start of the sweep, in DFT bins of a
    window of T seconds (App. A.2.1): the instantaneous rate of the true law
    (Eq. freqvst) at the band top against the linear rate a_1, times tau T."""
    T, _, a1 = chirp_model(f0, bw, k_dm, dm)
    nu_hi = f0 + 0.5 * bw
    rate_top = -0.5 * nu_hi ** 3 / (k_dm * dm)    # d nu / dt of Eq. freqvst at t = 0
    return abs(rate_top - a1) * tau * T


def fwhm_bins(N: int = 1 << 20) -> float:
    """Full width at half maximum of D_N^2 in bins, by bisection on the exact
    kernel (the paper's third-order estimate is 0.844, Eq. fwhm)."""
    lo, hi = 0.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if (dirichlet(mid, N) / N) ** 2 > 0.5:
            lo = mid
        else:
            hi = mid
    return 2.0 * lo
