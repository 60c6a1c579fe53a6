"""ctypes binding of the Chimageator pre-integrator on a uniform linear array
(the chirp_chimg_* entry points of include/chirp_gb300.h): argument
marshalling only, every step runs in the CUDA library.

The search (Sec. 4.2, App. B.2 of the paper) mixes every antenna pair, grids
equal spacings, takes a spatial DFT, integrates and dumps, and sums 2F+1
bins per dump along each trial chirp's trajectory (Eq. chimg_pth, Eq. eth).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _buf, _check, _stream_handle, load

__all__ = ["ChimgPlan", "Chimg2dPlan", "lines_run"]


class _ChimgConfig(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int), ("spacing_m", ctypes.c_double), ("f0_hz", ctypes.c_double),
                ("bw_hz", ctypes.c_double), ("k_dm", ctypes.c_double), ("n_samp", ctypes.c_longlong),
                ("dm", ctypes.POINTER(ctypes.c_double)), ("n_dm", ctypes.c_int),
                ("dump_len", ctypes.c_int), ("l_dir", ctypes.POINTER(ctypes.c_double)),
                ("n_pix", ctypes.c_int), ("n_spatial", ctypes.c_int), ("half_width", ctypes.c_int),
                ("weights", ctypes.c_int)]


class _Chimg2dConfig(ctypes.Structure):
    _fields_ = [("n_x", ctypes.c_int), ("n_y", ctypes.c_int), ("dx_m", ctypes.c_double),
                ("dy_m", ctypes.c_double), ("f0_hz", ctypes.c_double), ("bw_hz", ctypes.c_double),
                ("k_dm", ctypes.c_double), ("n_samp", ctypes.c_longlong),
                ("dm", ctypes.POINTER(ctypes.c_double)), ("n_dm", ctypes.c_int),
                ("dump_len", ctypes.c_int), ("pix_lm", ctypes.POINTER(ctypes.c_double)),
                ("n_pix", ctypes.c_int), ("n_spatial_x", ctypes.c_int),
                ("n_spatial_y", ctypes.c_int), ("half_width_x", ctypes.c_int),
                ("half_width_y", ctypes.c_int), ("weights", ctypes.c_int)]


def _lib():
    lib = load()
    if not getattr(lib, "_chimg_ready", False):
        vp, i = ctypes.c_void_p, ctypes.c_int
        lib.chirp_chimg_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_ChimgConfig), vp]
        lib.chirp_chimg_create.restype = i
        lib.chirp_chimg_query.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), vp]
        lib.chirp_chimg_query.restype = i
        lib.chirp_chimg_grid.argtypes = [vp, vp, i, vp, i]
        lib.chirp_chimg_grid.restype = i
        lib.chirp_chimg_run.argtypes = [vp, vp, i, vp, i]
        lib.chirp_chimg_run.restype = i
        lib.chirp_chimg_destroy.argtypes = [vp]
        lib.chirp_chimg_destroy.restype = None
        lib.chirp_chimg2d_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Chimg2dConfig),
                                             vp]
        lib.chirp_chimg2d_create.restype = i
        lib.chirp_chimg2d_query.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), vp,
                                            ctypes.POINTER(i)]
        lib.chirp_chimg2d_query.restype = i
        lib.chirp_chimg_lines_run.argtypes = [vp, ctypes.c_longlong, i, i, i, ctypes.c_double, i,
                                              ctypes.POINTER(ctypes.c_double), i,
                                              ctypes.POINTER(i), ctypes.POINTER(i), vp, vp]
        lib.chirp_chimg_lines_run.restype = i
        lib.chirp_chimg2d_grid.argtypes = [vp, vp, i, vp, i]
        lib.chirp_chimg2d_grid.restype = i
        lib.chirp_chimg2d_run.argtypes = [vp, vp, i, vp, i]
        lib.chirp_chimg2d_run.restype = i
        lib.chirp_chimg2d_destroy.argtypes = [vp]
        lib.chirp_chimg2d_destroy.restype = None
        lib._chimg_ready = True
    return lib


class ChimgPlan:
    """A Chimageator pre-integrator plan (chirp_chimg_create) for n_ant antennas
    at spacing_m along u.  grid() fills Y [n_dump, Ns] complex64; run() fills
    E [n_dm, n_dump, n_pix] float32."""

    def __init__(self, n_ant, spacing_m, f0, bw, n_samp, dms, dump_len, l_dir, n_spatial,
                 half_width=1, weights="natural", k_dm=0.0, stream=None):
        self._dms = np.ascontiguousarray(np.asarray(dms, np.float64).ravel())
        self._ld = np.ascontiguousarray(np.asarray(l_dir, np.float64).ravel())
        c = _ChimgConfig()
        c.n_ant, c.spacing_m = int(n_ant), float(spacing_m)
        c.f0_hz, c.bw_hz, c.k_dm = float(f0), float(bw), float(k_dm)
        c.n_samp = int(n_samp)
        c.dm = self._dms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.n_dm = len(self._dms)
        c.dump_len = int(dump_len)
        c.l_dir = self._ld.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.n_pix = len(self._ld)
        c.n_spatial, c.half_width = int(n_spatial), int(half_width)
        c.weights = {"natural": 0, "uniform": 1}[weights]
        self._h = ctypes.c_void_p()
        _check(_lib().chirp_chimg_create(ctypes.byref(self._h), ctypes.byref(c), _stream_handle(stream)))
        nd = ctypes.c_longlong()
        self.n_win = np.zeros(c.n_dm, np.int32)
        _check(_lib().chirp_chimg_query(self._h, ctypes.byref(nd), ctypes.c_void_p(self.n_win.ctypes.data)))
        self.n_dump, self.n_dm, self.n_pix, self.n_spatial = nd.value, c.n_dm, c.n_pix, c.n_spatial

    def grid(self, volt, Y) -> None:
        vp, vl, _k1 = _buf(volt, np.complex64, "volt")
        yp, yl, _k2 = _buf(Y, np.complex64, "Y")
        _check(_lib().chirp_chimg_grid(self._h, vp, vl, yp, yl))

    def run(self, volt, energy) -> None:
        vp, vl, _k1 = _buf(volt, np.complex64, "volt")
        ep, el, _k2 = _buf(energy, np.float32, "energy")
        _check(_lib().chirp_chimg_run(self._h, vp, vl, ep, el))

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib().chirp_chimg_destroy(self._h)
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


class Chimg2dPlan:
    """A Chimageator pre-integrator plan for a uniform rectangular array of
    n_x x n_y antennas (chirp_chimg2d_create).  grid() fills Y [n_dump, Nx, Ny]
    complex64; run() fills E [n_dm, n_dump, n_pix] float32."""

    def __init__(self, n_x, n_y, dx_m, dy_m, f0, bw, n_samp, dms, dump_len, pix_lm, n_spatial,
                 half_width=(1, 1), weights="natural", k_dm=0.0, stream=None):
        self._dms = np.ascontiguousarray(np.asarray(dms, np.float64).ravel())
        self._pix = np.ascontiguousarray(np.asarray(pix_lm, np.float64).reshape(-1, 2))
        c = _Chimg2dConfig()
        c.n_x, c.n_y, c.dx_m, c.dy_m = int(n_x), int(n_y), float(dx_m), float(dy_m)
        c.f0_hz, c.bw_hz, c.k_dm = float(f0), float(bw), float(k_dm)
        c.n_samp = int(n_samp)
        c.dm = self._dms.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.n_dm = len(self._dms)
        c.dump_len = int(dump_len)
        c.pix_lm = self._pix.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.n_pix = len(self._pix)
        c.n_spatial_x, c.n_spatial_y = int(n_spatial[0]), int(n_spatial[1])
        c.half_width_x, c.half_width_y = int(half_width[0]), int(half_width[1])
        c.weights = {"natural": 0, "uniform": 1}[weights]
        self._h = ctypes.c_void_p()
        _check(_lib().chirp_chimg2d_create(ctypes.byref(self._h), ctypes.byref(c),
                                           _stream_handle(stream)))
        nd = ctypes.c_longlong()
        ns = ctypes.c_int()
        self.n_win = np.zeros(c.n_dm, np.int32)
        _check(_lib().chirp_chimg2d_query(self._h, ctypes.byref(nd),
                                          ctypes.c_void_p(self.n_win.ctypes.data), ctypes.byref(ns)))
        self.n_dump, self.n_dm, self.n_pix = nd.value, c.n_dm, c.n_pix
        self.n_spatial = (c.n_spatial_x, c.n_spatial_y)
        self.n_spacing = ns.value

    def grid(self, volt, Y) -> None:
        vp, vl, _k1 = _buf(volt, np.complex64, "volt")
        yp, yl, _k2 = _buf(Y, np.complex64, "Y")
        _check(_lib().chirp_chimg2d_grid(self._h, vp, vl, yp, yl))

    def run(self, volt, energy) -> None:
        vp, vl, _k1 = _buf(volt, np.complex64, "volt")
        ep, el, _k2 = _buf(energy, np.float32, "energy")
        _check(_lib().chirp_chimg2d_run(self._h, vp, vl, ep, el))

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib().chirp_chimg2d_destroy(self._h)
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


def lines_run(Y, n_ant, n_spatial, dump_len, bw, half_width, rates, trial_lens, stream=None):
    """The partial-sum recursion of App. B.2.1 on the paper's own model
    (chirp_chimg_lines_run): Y is the complex64 CUDA tensor [n_dump][Ns] that
    ChimgPlan.grid writes with natural weights; rates[g] = fdot tau of line g
    (cycles per spacing per second); trial_lens[g] the window lengths (dumps)
    of its trials.  Returns E, a float32 CUDA tensor [n_trial][n_dump], trials
    in line order and, within a line, by ascending length."""
    import torch
    if not (isinstance(Y, torch.Tensor) and Y.is_cuda and Y.dtype == torch.complex64
            and Y.is_contiguous() and Y.dim() == 2 and Y.shape[1] == n_spatial):
        raise TypeError("Y must be a contiguous complex64 CUDA tensor [n_dump][n_spatial]")
    lens = [sorted(int(n) for n in tl) for tl in trial_lens]
    off = np.zeros(len(lens) + 1, np.int32)
    off[1:] = np.cumsum([len(tl) for tl in lens])
    flat = np.array([n for tl in lens for n in tl], np.int32)
    rt = np.ascontiguousarray(rates, np.float64)
    E = torch.empty((int(off[-1]), Y.shape[0]), dtype=torch.float32, device=Y.device)
    _check(_lib().chirp_chimg_lines_run(
        ctypes.c_void_p(Y.data_ptr()), Y.shape[0], int(n_ant), int(n_spatial), int(dump_len),
        float(bw), int(half_width), rt.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(lens),
        off.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        flat.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_void_p(E.data_ptr()),
        _stream_handle(stream)))
    return E
