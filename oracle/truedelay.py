"""FP64 numpy oracle of true-delay (wideband) beamforming of the dedispersed
voltages (test infrastructure only).

The phased beams of the hot path use one phase per antenna, exp(+2 pi j f0
tau_a) (narrowband; bandwidth smearing is part of that result).  True-delay
beams apply each antenna's geometric delay (Eq. tau3D) at every frequency:
in block b of the overlap-save grid, with X_ab the block's spectrum and H
the trial DM's chirp (Sec. 2.3.2),

    Y_pb(f) = H(f) sum_a exp(+2 pi j (f0 + f) tau_a(p)) X_ab(f),

and the beam is the inverse transform of Y_pb over the samples block b owns;
powers are |beam|^2 summed over each valid dump, as for the phased beams.
The block grid, the chirp (the C oracle's orc_chirp, baseband frequency of
bin b: b B / Nfft below Nfft/2, (b - Nfft) B / Nfft from there) and the
valid dumps are those of the hot path; block b owns t in
[b S + n_hi_max, (b+1) S + n_hi_max), block 0 also everything below and the
last block everything above.  Reading: the geometric delays (at most
B max|tau| samples) wrap circularly inside a block like the chirp's tail
does; the grid is not widened for them.
"""

from __future__ import annotations

import math

import numpy as np

import oracle

C_LIGHT = 299792458.0


def _freqs(nfft: int, bw: float) -> np.ndarray:
    b = np.arange(nfft)
    return np.where(b < nfft // 2, b, b - nfft) * bw / nfft


def _delays(xyz, l, m):
    n = math.sqrt(max(0.0, 1.0 - l * l - m * m))
    xyz = np.asarray(xyz, np.float64)
    return (xyz[:, 0] * l + xyz[:, 1] * m + xyz[:, 2] * (n - 1.0)) / C_LIGHT


def beams(x, xyz, pix_lm, f0, bw, k_dm, dms, nfft_min, dump_len) -> np.ndarray:
    """P[d][m][pix]: true-delay beam power summed over dump m (valid dumps only)."""
    x = np.asarray(x, np.complex128)
    n_ant, n_samp = x.shape
    n_dump = n_samp // dump_len
    P = np.zeros((len(dms), n_dump, len(pix_lm)))
    for d in range(len(dms)):
        lay = oracle.layout(dms, d, f0, bw, k_dm, n_samp, nfft_min)
        nfft, S, n_blk = lay["nfft"], lay["step"], lay["n_blk"]
        first, last = oracle.dump_range(n_samp, lay["n_hi"], lay["n_lo"], dump_len)
        if last < first:
            continue
        H = oracle.chirp(f0, bw, k_dm, dms[d], nfft)
        f = _freqs(nfft, bw)
        W = np.stack([np.exp(2j * math.pi * np.outer(f0 + f, _delays(xyz, l, m)))
                      for l, m in np.asarray(pix_lm, np.float64)])        # [pix][f][ant]
        t_lo, t_hi = first * dump_len, (last + 1) * dump_len
        pw = np.zeros((len(pix_lm), t_hi - t_lo))
        for b in range(n_blk):
            seg = np.zeros((n_ant, nfft), np.complex128)
            lo, hi = b * S, min(b * S + nfft, n_samp)
            seg[:, :hi - lo] = x[:, lo:hi]
            X = np.fft.fft(seg, axis=1)                                   # [ant][f]
            own_lo = 0 if b == 0 else b * S + lay["n_hi_max"]
            own_hi = n_samp if b == n_blk - 1 else (b + 1) * S + lay["n_hi_max"]
            a0, a1 = max(own_lo, t_lo), min(own_hi, t_hi)
            if a1 <= a0:
                continue
            for i in range(len(pix_lm)):
                Y = H * np.einsum("fa,af->f", W[i], X)
                y = np.fft.ifft(Y)
                pw[i, a0 - t_lo:a1 - t_lo] = np.abs(y[a0 - b * S:a1 - b * S]) ** 2
        sums = pw.reshape(len(pix_lm), last - first + 1, dump_len).sum(axis=2)
        P[d, first:last + 1] = sums.T
    return P
