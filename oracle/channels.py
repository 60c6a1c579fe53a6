"""FP64 numpy oracle of the combination of coarse channels (test infrastructure
only).

A wide band is searched as C coarse channels, each an independent search
about its own centre f_c with the same bandwidth B and dump length L (the
precision form's 8 x 42 MHz channels).  A channel's output at dump m refers
to arrivals at f_c (the time reference of Sec. 2.3.2's dedispersion about
the band centre), so a pulse reaches channel c later than the top channel
(f_ref = max f_c) by Eq. dmdelay:

    delta_c = k DM (f_c^-2 - f_ref^-2) seconds = delta_c B / L dumps.

Reading: the channels' powers are aligned to the top channel by
s_c = rint(delta_c B / L) dumps and added incoherently,

    E[d][m][pix] = sum_c P_c[d][m + s_c(d)][pix],

where every channel's dump m + s_c(d) exists and is valid for that DM
(first_c[d] <= m + s_c(d) <= last_c[d]); elsewhere E is zero.
"""

from __future__ import annotations

import numpy as np


def shifts(f_c, bw, L, k_dm, dms) -> np.ndarray:
    """s[d][c] = rint(k DM (f_c^-2 - f_ref^-2) B / L), f_ref = max f_c."""
    f_c = np.asarray(f_c, np.float64)
    f_ref = float(f_c.max())
    out = np.zeros((len(dms), len(f_c)), np.int64)
    for d, dm in enumerate(dms):
        for c, f in enumerate(f_c):
            out[d, c] = int(np.rint(k_dm * dm * (f ** -2 - f_ref ** -2) * bw / L))
    return out


def combine(P, first, last, f_c, bw, L, k_dm, dms) -> np.ndarray:
    """P: list over channels of [n_dm][n_dump][n_pix]; first/last: lists of
    [n_dm] valid-dump bounds per channel.  Returns E [n_dm][n_dump][n_pix]."""
    C = len(P)
    n_dm, n_dump, n_pix = np.asarray(P[0]).shape
    s = shifts(f_c, bw, L, k_dm, dms)
    E = np.zeros((n_dm, n_dump, n_pix))
    for d in range(n_dm):
        for m in range(n_dump):
            ok = True
            acc = np.zeros(n_pix)
            for c in range(C):
                mc = m + s[d, c]
                if mc >= n_dump or mc < first[c][d] or mc > last[c][d]:
                    ok = False
                    break
                acc += np.asarray(P[c][d][mc], np.float64)
            if ok:
                E[d, m] = acc
    return E


def channel_centres(f_mid: float, chan_bw: float, n_chan: int) -> np.ndarray:
    """Centres of n_chan adjacent channels of width chan_bw around f_mid."""
    return f_mid + (np.arange(n_chan) - (n_chan - 1) / 2.0) * chan_bw

