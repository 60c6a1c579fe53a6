"""ctypes binding of the Chirpolator pre-integrator (the chirp_cpi_* entry
points of include/chirp_gb300.h): argument marshalling only, every step runs
in the CUDA library.

The search (Sec. 3, App. A.3 of the paper) works on the raw voltages: pair
mixing (Eq. xpq), block-based sliding DFTs (Sec. A.3.2, Eq. block_cic) and
an image per trial DM from the 2F+1 bins around each pair's tone (Sec. 3.4,
Eqs. pth and eth).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import CHIRP_HOST, _buf, _check, _stream_handle, load

__all__ = ["CpiPlan", "CPI_STAGES"]

CPI_STAGES = ("moments", "partial", "cic", "image")


class _CpiConfig(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int), ("xyz_m", ctypes.POINTER(ctypes.c_double)),
                ("f0_hz", ctypes.c_double), ("bw_hz", ctypes.c_double),
                ("k_dm", ctypes.c_double), ("n_samp", ctypes.c_longlong),
                ("dm", ctypes.POINTER(ctypes.c_double)), ("n_dm", ctypes.c_int),
                ("blk_len", ctypes.c_int), ("pix_lm", ctypes.POINTER(ctypes.c_double)),
                ("n_pix", ctypes.c_int), ("half_width", ctypes.c_int), ("max_bin", ctypes.c_int),
                ("image_mode", ctypes.c_int)]


class _CpiInfo(ctypes.Structure):
    _fields_ = [("n_pair", ctypes.c_int), ("n_blk", ctypes.c_longlong), ("max_bin", ctypes.c_int),
                ("n_freq", ctypes.c_int), ("sub_len", ctypes.c_int), ("n_terms", ctypes.c_int),
                ("work_bytes", ctypes.c_longlong)]


def _lib():
    lib = load()
    if not getattr(lib, "_cpi_ready", False):
        vp, i = ctypes.c_void_p, ctypes.c_int
        lib.chirp_cpi_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_CpiConfig), vp]
        lib.chirp_cpi_create.restype = i
        lib.chirp_cpi_query.argtypes = [vp, ctypes.POINTER(_CpiInfo)]
        lib.chirp_cpi_query.restype = i
        lib.chirp_cpi_layout.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double), vp]
        lib.chirp_cpi_layout.restype = i
        lib.chirp_cpi_run.argtypes = [vp, vp, i, vp, i]
        lib.chirp_cpi_run.restype = i
        lib.chirp_cpi_spectra.argtypes = [vp, vp, i, vp, vp, i]
        lib.chirp_cpi_spectra.restype = i
        lib.chirp_cpi_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.chirp_cpi_timing.restype = i
        lib.chirp_cpi_destroy.argtypes = [vp]
        lib.chirp_cpi_destroy.restype = None
        lib._cpi_ready = True
    return lib


def _f64(a, shape_tail=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape_tail is not None and a.shape[1:] != shape_tail:
        raise ValueError("expected shape [n, %s]" % ", ".join(map(str, shape_tail)))
    return a


class CpiPlan:
    """A Chirpolator pre-integrator search plan (chirp_cpi_create).

    xyz [M, 3] metres; dms [n_dm] > 0; pix_lm [n_pix, 2]; blk_len L (power of
    two); half_width F; max_bin K (0: what the pixels need).  Outputs:
    run() fills E [n_dm, n_blk, n_pix] float32; spectra() fills V and X
    [n_dm, n_blk, 2K+1, n_pair] complex64."""

    def __init__(self, xyz, f0, bw, n_samp, dms, blk_len, pix_lm, half_width=2, max_bin=0,
                 k_dm=0.0, stream=None, image_mode=0):
        self._xyz = _f64(xyz, (3,))
        self._dms = _f64(dms).ravel()
        self._pix = _f64(pix_lm, (2,))
        c = _CpiConfig()
        c.n_ant = self._xyz.shape[0]
        c.xyz_m = self._xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.f0_hz, c.bw_hz, c.k_dm = float(f0), float(bw), float(k_dm)
        c.n_samp = int(n_samp)
        c.dm = self._dms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.n_dm = len(self._dms)
        c.blk_len = int(blk_len)
        c.pix_lm = self._pix.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.n_pix = self._pix.shape[0]
        c.half_width, c.max_bin = int(half_width), int(max_bin)
        c.image_mode = int(image_mode)  # 0: tensor cores (dense filter), 1: CUDA-core gathers
        self._h = ctypes.c_void_p()
        _check(_lib().chirp_cpi_create(ctypes.byref(self._h), ctypes.byref(c), _stream_handle(stream)))
        inf = _CpiInfo()
        _check(_lib().chirp_cpi_query(self._h, ctypes.byref(inf)))
        self.info = {k: getattr(inf, k) for k, _ in _CpiInfo._fields_}
        self.n_ant, self.n_samp, self.n_dm = c.n_ant, c.n_samp, c.n_dm
        self.n_pix, self.n_pair, self.n_blk = c.n_pix, inf.n_pair, inf.n_blk
        self.max_bin = inf.max_bin

    def layout(self, d: int) -> dict:
        nw, fd = ctypes.c_int(), ctypes.c_double()
        kb = np.zeros(self.n_pair, np.int32)
        _check(_lib().chirp_cpi_layout(self._h, int(d), ctypes.byref(nw), ctypes.byref(fd),
                                       ctypes.c_void_p(kb.ctypes.data)))
        return {"n_win": nw.value, "fdot": fd.value, "pair_bins": kb}

    def run(self, volt, energy) -> None:
        vp, vl, _k1 = _buf(volt, np.complex64, "volt")
        ep, el, _k2 = _buf(energy, np.float32, "energy")
        _check(_lib().chirp_cpi_run(self._h, vp, vl, ep, el))

    def spectra(self, volt, V=None, X=None) -> None:
        vp, vl, _k1 = _buf(volt, np.complex64, "volt")
        locs, ptrs, keep = set(), [], []
        for a, nm in ((V, "V"), (X, "X")):
            if a is None:
                ptrs.append(None)
                continue
            p, loc, k = _buf(a, np.complex64, nm)
            ptrs.append(p)
            locs.add(loc)
            keep.append(k)
        if len(locs) > 1:
            raise TypeError("V and X must both be on the host or both on the device")
        loc = locs.pop() if locs else CHIRP_HOST
        _check(_lib().chirp_cpi_spectra(self._h, vp, vl, ptrs[0], ptrs[1], loc))

    def timing(self) -> dict:
        ms = (ctypes.c_double * 4)()
        _check(_lib().chirp_cpi_timing(self._h, ms))
        return dict(zip(CPI_STAGES, list(ms)))

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib().chirp_cpi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



