"""FP64 CPU oracle of the coherent-dedispersion pulse search (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it.  The arithmetic lives in ``chirp_oracle.c`` (plain C,
FP64); this module compiles it with gcc on first use and wraps it with ctypes.

Conventions: complex arrays are numpy complex128, antenna-major [n_ant, n_samp];
the DM list is in pc cm^-3; frequencies in Hz; k_dm in s Hz^2 / (pc cm^-3).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chirp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_llp = ctypes.POINTER(ctypes.c_longlong)
_ip = ctypes.POINTER(ctypes.c_int)
_ll = ctypes.c_longlong
_d = ctypes.c_double
_i = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile chirp_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
           "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_fft.argtypes = [_dp, _ll, _i]
            lib.orc_fft.restype = _i
            lib.orc_dft.argtypes = [_dp, _dp, _ll, _i]
            lib.orc_sweep.argtypes = [_d, _d, _d, _d, _llp, _llp]
            lib.orc_nfft_for_dm.argtypes = [_d, _d, _d, _d, _ll, _ll]
            lib.orc_nfft_for_dm.restype = _ll
            lib.orc_layout.argtypes = [_dp, _i, _i, _d, _d, _d, _ll, _ll, _llp]
            lib.orc_layout.restype = _i
            lib.orc_dump_range.argtypes = [_ll, _ll, _ll, _i, _llp, _llp]
            lib.orc_chirp.argtypes = [_d, _d, _d, _d, _ll, _dp]
            lib.orc_dedisperse_span.argtypes = [_dp, _i, _ll, _d, _d, _d, _dp, _i, _i, _ll,
                                                _ll, _ll, _dp]
            lib.orc_dedisperse_span.restype = _i
            lib.orc_correlate.argtypes = [_dp, _i, _ll, _i, _ll, _ll, _ll, _ll, _dp]
            lib.orc_beam_weights.argtypes = [_dp, _i, _dp, _i, _d, _dp]
            lib.orc_beamform.argtypes = [_dp, _i, _ll, _i, _ll, _ll, _ll, _ll, _dp, _i, _dp]
            lib.orc_chirpolator.argtypes = [_dp, _i, _ll, _d, _d, _d, _dp, _i, _ll, _i, _ip, _i,
                                            _ll, _ll, _dp]
            lib.orc_chirpolator.restype = _i
            lib.orc_chimageator.argtypes = [_dp, _i, _ll, _d, _d, _d, _dp, _i, _ll, _i, _dp, _dp,
                                            _i, _ip, _i, _ll, _ll, _dp]
            lib.orc_chimageator.restype = _i
            lib.orc_num_threads.restype = _i
            lib.orc_filterbank.argtypes = [_dp, _i, _ll, _i, _i, _dp]
            lib.orc_channel_shift.argtypes = [_d, _d, _d, _d, _i, _i, _i]
            lib.orc_channel_shift.restype = _ll
            _fp = ctypes.POINTER(ctypes.c_float)
            lib.orc_series_stats.argtypes = [_fp, _i, _ll, _i, _llp, _llp, _fp]
            lib.orc_detect.argtypes = [_fp, _i, _ll, _i, _llp, _llp, ctypes.c_float, _fp, _ip,
                                       _llp, _ip, _fp, _ll]
            lib.orc_detect.restype = _ll
            lib.orc_incoherent.argtypes = [_dp, _i, _ll, _d, _d, _d, _i, _dp, _i, _dp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- wrappers
def num_threads() -> int:
    return int(_load().orc_num_threads())


def fft(x, sign: int = -1) -> np.ndarray:
    """Radix-2 FFT, unnormalised, exp(sign 2 pi j n k / N)."""
    y = _c128(x).copy()
    rc = _load().orc_fft(_ptr(y), y.size, sign)
    if rc:
        raise ValueError("orc_fft: length %d is not a power of two" % y.size)
    return y


def dft(x, sign: int = -1) -> np.ndarray:
    """Direct O(N^2) DFT, exp(sign 2 pi j n k / N)."""
    xx = _c128(x)
    out = np.empty_like(xx)
    _load().orc_dft(_ptr(xx), _ptr(out), xx.size, sign)
    return out


def sweep(f0, bw, k_dm, dm):
    """(n_hi, n_lo) dispersion sweep in samples above / below f0."""
    hi, lo = ctypes.c_longlong(), ctypes.c_longlong()
    _load().orc_sweep(f0, bw, k_dm, dm, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def nfft_for_dm(f0, bw, k_dm, dm, n_samp, nfft_min) -> int:
    return int(_load().orc_nfft_for_dm(f0, bw, k_dm, dm, n_samp, nfft_min))


def layout(dms, d, f0, bw, k_dm, n_samp, nfft_min) -> dict:
    """Block grid of DM number d: nfft, n_hi, n_lo, n_hi_max, n_lo_max, step, n_blk."""
    dd = _f64(dms)
    out = np.zeros(7, dtype=np.int64)
    rc = _load().orc_layout(_ptr(dd), dd.size, d, f0, bw, k_dm, n_samp, nfft_min,
                            _ptr(out, ctypes.c_longlong))
    if rc:
        raise ValueError("orc_layout failed (%d)" % rc)
    keys = ("nfft", "n_hi", "n_lo", "n_hi_max", "n_lo_max", "step", "n_blk")
    return {k: int(v) for k, v in zip(keys, out)}


def dump_range(n_samp, n_hi, n_lo, dump_len):
    first, last = ctypes.c_longlong(), ctypes.c_longlong()
    _load().orc_dump_range(n_samp, n_hi, n_lo, dump_len, ctypes.byref(first), ctypes.byref(last))
    return first.value, last.value


def chirp(f0, bw, k_dm, dm, nfft) -> np.ndarray:
    """H_DM at the nfft bins (natural FFT order)."""
    H = np.empty(nfft, dtype=np.complex128)
    _load().orc_chirp(f0, bw, k_dm, dm, nfft, _ptr(H))
    return H


def dedisperse(x, f0, bw, k_dm, dms, d, nfft_min, t_lo=0, t_hi=None) -> np.ndarray:
    """Dedispersed voltages [n_ant, t_hi - t_lo] of DM number d (zero where invalid)."""
    xx = _c128(np.atleast_2d(x))
    n_ant, n_samp = xx.shape
    t_hi = n_samp if t_hi is None else t_hi
    dd = _f64(dms)
    y = np.empty((n_ant, t_hi - t_lo), dtype=np.complex128)
    rc = _load().orc_dedisperse_span(_ptr(xx), n_ant, n_samp, f0, bw, k_dm, _ptr(dd), dd.size,
                                     d, nfft_min, t_lo, t_hi, _ptr(y))
    if rc:
        raise ValueError("orc_dedisperse_span failed (%d)" % rc)
    return y


def correlate(y, dump_len, m0, m1, first, last) -> np.ndarray:
    yy = _c128(y)
    n_ant, span = yy.shape
    V = np.empty((m1 - m0, n_ant * (n_ant + 1) // 2), dtype=np.complex128)
    _load().orc_correlate(_ptr(yy), n_ant, span, dump_len, m0, m1, first, last, _ptr(V))
    return V


def beam_weights(xyz, pix_lm, f0) -> np.ndarray:
    xx, pp = _f64(xyz), _f64(pix_lm)
    W = np.empty((pp.shape[0], xx.shape[0]), dtype=np.complex128)
    _load().orc_beam_weights(_ptr(xx), xx.shape[0], _ptr(pp), pp.shape[0], f0, _ptr(W))
    return W


def beamform(y, W, dump_len, m0, m1, first, last) -> np.ndarray:
    yy, WW = _c128(y), _c128(W)
    n_ant, span = yy.shape
    P = np.empty((m1 - m0, WW.shape[0]), dtype=np.float64)
    _load().orc_beamform(_ptr(yy), n_ant, span, dump_len, m0, m1, first, last, _ptr(WW),
                         WW.shape[0], _ptr(P))
    return P


def chirpolator(x, f0, bw, k_dm, dms, nfft_min, dump_len, d_sel=None, m0=0, m1=None):
    """Visibilities [n_sel, m1-m0, n_ant(n_ant+1)/2] complex128."""
    xx = _c128(x)
    n_ant, n_samp = xx.shape
    dd = _f64(dms)
    sel = np.arange(dd.size, dtype=np.int32) if d_sel is None else np.asarray(d_sel, np.int32)
    m1 = n_samp // dump_len if m1 is None else m1
    V = np.empty((sel.size, m1 - m0, n_ant * (n_ant + 1) // 2), dtype=np.complex128)
    rc = _load().orc_chirpolator(_ptr(xx), n_ant, n_samp, f0, bw, k_dm, _ptr(dd), dd.size,
                                 nfft_min, dump_len, _ptr(sel, ctypes.c_int), sel.size, m0, m1,
                                 _ptr(V))
    if rc:
        raise ValueError("orc_chirpolator failed (%d)" % rc)
    return V


def chimageator(x, f0, bw, k_dm, dms, nfft_min, dump_len, xyz, pix_lm, d_sel=None, m0=0,
                m1=None):
    """Beam powers [n_sel, m1-m0, n_pix] float64."""
    xx = _c128(x)
    n_ant, n_samp = xx.shape
    dd, xz, pp = _f64(dms), _f64(xyz), _f64(pix_lm)
    sel = np.arange(dd.size, dtype=np.int32) if d_sel is None else np.asarray(d_sel, np.int32)
    m1 = n_samp // dump_len if m1 is None else m1
    P = np.empty((sel.size, m1 - m0, pp.shape[0]), dtype=np.float64)
    rc = _load().orc_chimageator(_ptr(xx), n_ant, n_samp, f0, bw, k_dm, _ptr(dd), dd.size,
                                 nfft_min, dump_len, _ptr(xz), _ptr(pp), pp.shape[0],
                                 _ptr(sel, ctypes.c_int), sel.size, m0, m1, _ptr(P))
    if rc:
        raise ValueError("orc_chimageator failed (%d)" % rc)
    return P


def filterbank(x, n_chan, n_int) -> np.ndarray:
    """Power-beam filterbank S [n_chan, T_fb] (ascending channel frequency)."""
    xx = _c128(np.atleast_2d(x))
    n_ant, n_samp = xx.shape
    T = n_samp // (n_chan * n_int)
    S = np.empty((n_chan, T), dtype=np.float64)
    _load().orc_filterbank(_ptr(xx), n_ant, n_samp, n_chan, n_int, _ptr(S))
    return S


def channel_shift(f0, bw, k_dm, dm, n_chan, n_int, c) -> int:
    return int(_load().orc_channel_shift(f0, bw, k_dm, dm, n_chan, n_int, c))


def incoherent(S, f0, bw, k_dm, n_int, dms) -> np.ndarray:
    """Incoherent dedispersion D [n_dm, T_fb] of a filterbank S [n_chan, T_fb]."""
    SS = _f64(S)
    n_chan, T = SS.shape
    dd = _f64(dms)
    D = np.empty((dd.size, T), dtype=np.float64)
    _load().orc_incoherent(_ptr(SS), n_chan, T, f0, bw, k_dm, n_int, _ptr(dd), dd.size, _ptr(D))
    return D


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def series_stats(P, first, last) -> np.ndarray:
    """(median, 1.4826 MAD) [n_dm, n_pix, 2] of every (DM, pixel) series of
    dump powers P [n_dm, n_dump, n_pix] over the valid dumps, in FP32."""
    PP = _f32(P)
    n_dm, n_dump, n_pix = PP.shape
    f = np.ascontiguousarray(first, dtype=np.int64)
    l = np.ascontiguousarray(last, dtype=np.int64)
    st = np.empty((n_dm, n_pix, 2), np.float32)
    _load().orc_series_stats(_fptr(PP), n_dm, n_dump, n_pix, f.ctypes.data_as(_llp),
                             l.ctypes.data_as(_llp), _fptr(st))
    return st


def detect(P, first, last, snr_min):
    """Candidates (local S/N maxima >= snr_min) of P [n_dm, n_dump, n_pix]:
    (d int32 [n], m int64 [n], p int32 [n], snr float32 [n]) in (d, m, p) order."""
    PP = _f32(P)
    n_dm, n_dump, n_pix = PP.shape
    f = np.ascontiguousarray(first, dtype=np.int64)
    l = np.ascontiguousarray(last, dtype=np.int64)
    st = series_stats(PP, f, l)
    cap = 1 << 16
    while True:
        cd = np.empty(cap, np.int32)
        cm = np.empty(cap, np.int64)
        cp = np.empty(cap, np.int32)
        cs = np.empty(cap, np.float32)
        n = _load().orc_detect(_fptr(PP), n_dm, n_dump, n_pix, f.ctypes.data_as(_llp),
                               l.ctypes.data_as(_llp), float(snr_min), _fptr(st),
                               cd.ctypes.data_as(_ip), cm.ctypes.data_as(_llp),
                               cp.ctypes.data_as(_ip), _fptr(cs), cap)
        if n <= cap:
            return cd[:n], cm[:n], cp[:n], cs[:n]
        cap = int(n)
