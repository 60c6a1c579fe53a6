"""Error metrics shared by the GPU-vs-oracle parity tests.

Visibilities: max |V_gpu - V_oracle| / sqrt(V_pp V_qq) over valid dumps and
pairs.  Beam powers: max |P_gpu - P_oracle| / P_oracle over valid dumps.
Dedispersed voltages: rms and max of |y_gpu - y_oracle| over rms(y_oracle).

FP32 budget (the tolerance the FP32 path is held to): visibilities and beam
powers 1e-5.  For the voltages themselves the bound follows from the
arithmetic: two FP32 transforms of length N contribute ~eps*sqrt(log2 N) each
(eps = 6e-8) and the FP32 chirp phase ~2e-7 rad, so the rms relative error
is ~1e-6; we allow 3e-6 rms and 4e-5 max (tail of ~1e7 samples).
"""
import numpy as np

TOL_VIS = 1e-5
TOL_POW = 1e-5
TOL_Y_RMS = 3e-6
TOL_Y_MAX = 4e-5


def pair_index(n_ant):
    return [(p, q) for p in range(n_ant) for q in range(p, n_ant)]


def vis_error(V_gpu, V_orc, n_ant):
    pairs = pair_index(n_ant)
    autos = np.array([pairs.index((a, a)) for a in range(n_ant)])
    vii = np.abs(V_orc[..., autos].real)                 # [.., n_ant]
    p_idx = np.array([p for p, _ in pairs])
    q_idx = np.array([q for _, q in pairs])
    norm = np.sqrt(vii[..., p_idx] * vii[..., q_idx])
    valid = norm > 0
    err = np.abs(V_gpu.astype(np.complex128) - V_orc)
    if not valid.any():
        return 0.0
    return float((err[valid] / norm[valid]).max())


def pow_error(P_gpu, P_orc):
    valid = P_orc > 0
    if not valid.any():
        return 0.0
    return float((np.abs(P_gpu.astype(np.float64) - P_orc)[valid] / P_orc[valid]).max())


def y_error(y_gpu, y_orc):
    d = np.abs(y_gpu.astype(np.complex128) - y_orc)
    ref = np.sqrt(np.mean(np.abs(y_orc) ** 2))
    if ref == 0:
        return 0.0, float(d.max())
    return float(np.sqrt(np.mean(d ** 2)) / ref), float(d.max() / ref)
