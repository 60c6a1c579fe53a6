"""GB300 (sm_103a) coherent-dedispersion pulse search: Python binding.

A thin ctypes layer over ``libchirp_gb300.so`` (C ABI in include/chirp_gb300.h).
It only marshals arguments: every step of the search runs in the library's
CUDA kernels.  There is no CPU fallback; if the library is missing or cannot
load, every entry point raises.

Buffers may be torch tensors (CUDA tensors are passed as device pointers, CPU
tensors as host pointers) or numpy arrays (host).  Voltages are complex64
[n_ant, n_samp]; visibilities complex64 [n_dm, n_dump, n_pair]; beam powers
float32 [n_dm, n_dump, n_pix].

Paper: Bannister & Cornwell, "The Chirpolator & The Chimageator"
(arXiv:1109.3186).  Dedispersion: Sec. 2.3.2 with Eq. 1; correlation:
Eq. xpq's p.q^* products integrated per dump; beams: Sec. 2.4.2 with Eq. tau3D.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["Plan", "PropNet", "load", "build", "CHIRP_HOST", "CHIRP_DEVICE", "BEAM_AUTO", "BEAM_FP32_SIMT",
           "BEAM_TC_3XBF16", "BEAM_VIS", "ChirpError", "chirp_plan_create", "chirp_plan_destroy",
           "chirp_combine_channels",
           "chirpolator_run", "chimageator_run", "chirp_dedisperse_run", "chirp_last_error",
           "EXPORTED_SYMBOLS"]

CHIRP_HOST, CHIRP_DEVICE = 0, 1
BEAM_AUTO, BEAM_FP32_SIMT, BEAM_TC_3XBF16, BEAM_VIS, BEAM_TC_BF16, BEAM_VIS_BF16 = 0, 1, 2, 3, 4, 5
IN_C64, IN_CI8 = 0, 1
CORR_AUTO, CORR_FP32_SIMT, CORR_TC_3XBF16, CORR_TC_BF16 = 0, 1, 2, 3
FLAG_GRAPHS, FLAG_AUTOTUNE, FLAG_LEAN = 1, 2, 4
TIMING_SELECT = 0x40000000  # chirp_stage_timing: time only the stages in the mask
CHIRP_OK, CHIRP_EINVAL, CHIRP_ENOMEM, CHIRP_ECUDA, CHIRP_ETIMEOUT, CHIRP_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
K_DM_DEFAULT = 4.148808e15

EXPORTED_SYMBOLS = ("chirp_plan_create", "chirp_plan_destroy", "chirp_plan_query",
                    "chirp_dm_layout", "chirp_dump_range", "chirp_dedisperse_run",
                    "chirpolator_run", "chimageator_run", "chirp_stage_timing",
                    "chirp_plan_status", "chirp_incoherent_run", "chirp_propnet_create",
                    "chirp_propnet_destroy", "chirp_propnet_param_count",
                    "chirp_propnet_set_params", "chirp_propnet_get_params",
                    "chirp_propnet_get_grads", "chirp_propnet_forward", "chirp_propnet_backward",
                    "chirp_propnet_train_step", "chirp_propnet_normalize", "chirp_propose_windows",
                    "chirpolator_run_selective", "chimageator_run_selective", "chirp_batch_run", "chirp_plan_fft_split", "chirp_detect",
                    "chirp_dedisperse_noalloc", "chirp_watchdog_selftest", "chirp_propnet_get_state",
                    "chirp_propnet_set_state", "chirp_last_error", "chirp_cpi_create",
                    "chirp_cpi_query", "chirp_cpi_layout", "chirp_cpi_run", "chirp_cpi_spectra",
                    "chirp_cpi_timing", "chirp_cpi_destroy", "chirp_chimg_create",
                    "chirp_chimg_query", "chirp_chimg_grid", "chirp_chimg_run",
                    "chirp_chimg_destroy", "chirp_chimg_lines_run", "chirp_combine_channels",
                    "chirp_chimg2d_create",
                    "chirp_chimg2d_query", "chirp_chimg2d_grid", "chirp_chimg2d_run",
                    "chirp_chimg2d_destroy", "chirp_truedelay_run")
STAGES = ("forward", "inv_rows", "inv_cols", "correlate", "beamform", "split", "chirp",
          "incoherent", "detect", "td_spectra")


class ChirpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("chirp error %d: %s" % (code, msg))
        self.code = code


class _Config(ctypes.Structure):
    _fields_ = [("n_ant", ctypes.c_int), ("xyz_m", ctypes.POINTER(ctypes.c_double)),
                ("f0_hz", ctypes.c_double), ("bw_hz", ctypes.c_double),
                ("k_dm", ctypes.c_double), ("n_samp", ctypes.c_longlong),
                ("dm", ctypes.POINTER(ctypes.c_double)), ("n_dm", ctypes.c_int),
                ("dump_len", ctypes.c_int), ("nfft_min", ctypes.c_longlong),
                ("pix_lm", ctypes.POINTER(ctypes.c_double)), ("n_pix", ctypes.c_int),
                ("beam_mode", ctypes.c_int), ("fb_chan", ctypes.c_int), ("fb_int", ctypes.c_int),
                ("fb_dm", ctypes.POINTER(ctypes.c_double)), ("fb_n_dm", ctypes.c_int),
                ("flags", ctypes.c_int), ("in_type", ctypes.c_int),
                ("in_scale", ctypes.POINTER(ctypes.c_float)), ("corr_mode", ctypes.c_int),
                ("beam_shape", ctypes.c_int),
                ("fft_row", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("n_dump", ctypes.c_longlong), ("n_pair", ctypes.c_int),
                ("n_group", ctypes.c_int), ("workspace_bytes", ctypes.c_longlong),
                ("ifft_points", ctypes.c_longlong), ("valid_samples", ctypes.c_longlong),
                ("beam_mode", ctypes.c_int), ("fb_samples", ctypes.c_longlong),
                ("beam_shape", ctypes.c_int), ("corr_mode", ctypes.c_int),
                ("dm_chunk", ctypes.c_int)]


_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load():
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB_PATH
        if not _build.up_to_date():
            path = _build.build()
        lib = ctypes.CDLL(path)
        vp, i, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
        lib.chirp_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(_Config), vp]
        lib.chirp_plan_create.restype = i
        lib.chirp_plan_destroy.argtypes = [vp]
        lib.chirp_plan_destroy.restype = None
        lib.chirp_plan_query.argtypes = [vp, ctypes.POINTER(_Info)]
        lib.chirp_plan_query.restype = i
        lib.chirp_dm_layout.argtypes = [vp, i, ctypes.POINTER(ll)]
        lib.chirp_dm_layout.restype = i
        lib.chirp_dump_range.argtypes = [vp, ctypes.POINTER(ll), ctypes.POINTER(ll)]
        lib.chirp_dump_range.restype = i
        lib.chirp_dedisperse_run.argtypes = [vp, vp, i, i, vp, i]
        lib.chirp_dedisperse_run.restype = i
        lib.chirpolator_run.argtypes = [vp, vp, i, vp, i]
        lib.chirpolator_run.restype = i
        lib.chimageator_run.argtypes = [vp, vp, i, vp, i]
        lib.chimageator_run.restype = i
        lib.chirp_truedelay_run.argtypes = [vp, vp, i, vp, i]
        lib.chirp_truedelay_run.restype = i
        lib.chirp_stage_timing.argtypes = [vp, i, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ll)]
        lib.chirp_stage_timing.restype = i
        lib.chirp_incoherent_run.argtypes = [vp, vp, i, vp, vp, i]
        lib.chirp_incoherent_run.restype = i
        fp = ctypes.POINTER(ctypes.c_float)
        lib.chirp_propnet_create.argtypes = [ctypes.POINTER(vp), i, i, i, i, i, i, vp]
        lib.chirp_propnet_create.restype = i
        lib.chirp_propnet_destroy.argtypes = [vp]
        lib.chirp_propnet_destroy.restype = None
        lib.chirp_propnet_param_count.argtypes = [vp]
        lib.chirp_propnet_param_count.restype = ll
        for nm in ("chirp_propnet_set_params", "chirp_propnet_get_params", "chirp_propnet_get_grads"):
            getattr(lib, nm).argtypes = [vp, fp]
            getattr(lib, nm).restype = i
        lib.chirp_propnet_get_state.argtypes = [vp, fp, fp, fp, ctypes.POINTER(ll)]
        lib.chirp_propnet_get_state.restype = i
        lib.chirp_propnet_set_state.argtypes = [vp, fp, fp, fp, ll]
        lib.chirp_propnet_set_state.restype = i
        lib.chirp_propnet_forward.argtypes = [vp, vp, i, vp]
        lib.chirp_propnet_forward.restype = i
        lib.chirp_propnet_backward.argtypes = [vp, vp, vp, i, ctypes.c_float, fp]
        lib.chirp_propnet_backward.restype = i
        lib.chirp_propnet_train_step.argtypes = [vp, vp, vp, i, ctypes.c_float, ctypes.c_float, fp]
        lib.chirp_propnet_train_step.restype = i
        lib.chirp_propnet_normalize.argtypes = [vp, i, ll, vp, vp]
        lib.chirp_propnet_normalize.restype = i
        lib.chirp_propose_windows.argtypes = [vp, i, ll, i, ctypes.c_float, vp, vp]
        lib.chirp_propose_windows.restype = i
        lib.chirpolator_run_selective.argtypes = [vp, vp, i, vp, vp, i]
        lib.chirpolator_run_selective.restype = i
        lib.chimageator_run_selective.argtypes = [vp, vp, i, vp, vp, i]
        lib.chimageator_run_selective.restype = i
        lib.chirp_batch_run.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i),
                                        ctypes.POINTER(vp), ctypes.POINTER(i), ctypes.POINTER(i), i]
        lib.chirp_batch_run.restype = i
        lib.chirp_plan_fft_split.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(i), ctypes.POINTER(i)]
        lib.chirp_plan_fft_split.restype = i
        lib.chirp_detect.argtypes = [vp, vp, i, ctypes.c_float, vp, ctypes.c_longlong, i,
                                     ctypes.POINTER(ctypes.c_longlong), vp]
        lib.chirp_detect.restype = i
        lib.chirp_plan_status.argtypes = [vp]
        lib.chirp_plan_status.restype = i
        lib.chirp_dedisperse_noalloc.argtypes = [vp, i, ll, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_double, ll, vp, vp]
        lib.chirp_dedisperse_noalloc.restype = i
        lib.chirp_watchdog_selftest.argtypes = [ctypes.c_uint, ctypes.POINTER(ctypes.c_double), vp]
        lib.chirp_watchdog_selftest.restype = i
        dp = ctypes.POINTER(ctypes.c_double)
        llp = ctypes.POINTER(ll)
        lib.chirp_combine_channels.argtypes = [ctypes.POINTER(vp), i, i, ll, i, llp, llp, dp,
                                               ctypes.c_double, i, ctypes.c_double, dp, vp, vp]
        lib.chirp_combine_channels.restype = i
        lib.chirp_last_error.argtypes = []
        lib.chirp_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        raise ChirpError(rc, load().chirp_last_error().decode(errors="replace"))


def _buf(a, dtype_np, what: str):
    """(pointer, location, keepalive) of a torch tensor or numpy array."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        want = {np.complex64: torch.complex64, np.float32: torch.float32}[dtype_np]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError("%s must be a contiguous %s tensor" % (what, want))
        return ctypes.c_void_p(a.data_ptr()), (CHIRP_DEVICE if a.is_cuda else CHIRP_HOST), a
    arr = np.asarray(a)
    if arr.dtype != dtype_np or not arr.flags["C_CONTIGUOUS"]:
        raise TypeError("%s must be a C-contiguous %s array" % (what, np.dtype(dtype_np).name))
    return ctypes.c_void_p(arr.ctypes.data), CHIRP_HOST, arr


class Candidate(ctypes.Structure):
    """chirp_candidate: one detection (trial DM index, dump, pixel, S/N, power)."""
    _fields_ = [("dump", ctypes.c_longlong), ("dm", ctypes.c_int), ("pix", ctypes.c_int),
                ("snr", ctypes.c_float), ("power", ctypes.c_float)]


CANDIDATE_DTYPE = np.dtype([("dump", np.int64), ("dm", np.int32), ("pix", np.int32),
                            ("snr", np.float32), ("power", np.float32)])


def _vbuf(a, in_type=None):
    """_buf of a voltage input: complex64 [M, N], or complex int8 as int8
    [M, N, 2] (in_type None accepts either)."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        is_i8 = a.dtype == torch.int8
    else:
        is_i8 = np.asarray(a).dtype == np.int8
    if in_type is not None and is_i8 != (in_type == IN_CI8):
        raise TypeError("volt must be %s for this plan"
                        % ("int8 [n_ant, n_samp, 2]" if in_type == IN_CI8 else "complex64"))
    if not is_i8:
        return _buf(a, np.complex64, "volt")
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise TypeError("volt must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), (CHIRP_DEVICE if a.is_cuda else CHIRP_HOST), a
    arr = np.asarray(a)
    if not arr.flags["C_CONTIGUOUS"]:
        raise TypeError("volt must be C-contiguous")
    return ctypes.c_void_p(arr.ctypes.data), CHIRP_HOST, arr


def _stream_handle(stream):
    if stream is not None:
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:  # pragma: no cover
        pass
    return ctypes.c_void_p(0)


# ------------------------------------------------------------ raw C-ABI names
def chirp_plan_create(cfg: _Config, stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load().chirp_plan_create(ctypes.byref(h), ctypes.byref(cfg), _stream_handle(stream)))
    return h


def chirp_plan_destroy(h) -> None:
    load().chirp_plan_destroy(h)


def chirp_dedisperse_run(h, volt, d: int, y_out, in_type=None) -> None:
    vp, vl, _k1 = _vbuf(volt, in_type)
    yp, yl, _k2 = _buf(y_out, np.complex64, "y_out")
    _check(load().chirp_dedisperse_run(h, vp, vl, int(d), yp, yl))


def chirpolator_run(h, volt, vis_out, in_type=None) -> None:
    vp, vl, _k1 = _vbuf(volt, in_type)
    op, ol, _k2 = _buf(vis_out, np.complex64, "vis_out")
    _check(load().chirpolator_run(h, vp, vl, op, ol))


def chimageator_run(h, volt, pow_out, in_type=None) -> None:
    vp, vl, _k1 = _vbuf(volt, in_type)
    op, ol, _k2 = _buf(pow_out, np.float32, "pow_out")
    _check(load().chimageator_run(h, vp, vl, op, ol))


def chirp_dedisperse_noalloc(volt, f0: float, bw: float, k_dm: float, dm: float,
                             nfft_min: int, y_out, stream=None) -> None:
    """Allocation-free one-DM dedispersion (device buffers only); see the
    header for who needs it, its scratch limit and its set-up call."""
    vp, vl, _k1 = _buf(volt, np.complex64, "volt")
    yp, yl, _k2 = _buf(y_out, np.complex64, "y_out")
    if vl != CHIRP_DEVICE or yl != CHIRP_DEVICE:
        raise TypeError("chirp_dedisperse_noalloc takes device buffers only")
    n_ant, n_samp = volt.shape
    _check(load().chirp_dedisperse_noalloc(vp, int(n_ant), int(n_samp), float(f0), float(bw),
                                           float(k_dm), float(dm), int(nfft_min), yp,
                                           _stream_handle(stream)))


def chirp_watchdog_selftest(polls: int = 1 << 16, stream=None):
    """Run the device watchdog's self-test (a bounded wait on a barrier that
    nothing arrives at); returns (status code, kernel milliseconds).  The
    expected code is CHIRP_ETIMEOUT."""
    ms = ctypes.c_double(0.0)
    rc = load().chirp_watchdog_selftest(int(polls), ctypes.byref(ms), _stream_handle(stream))
    return int(rc), float(ms.value)


def chirp_batch_run(plans, volts, outs, backends) -> None:
    """Queue several searches (chirp_batch_run); backends: 0 Chirpolator, 1 Chimageator."""
    n = len(plans)
    keep = []
    vp = (ctypes.c_void_p * n)()
    vl = (ctypes.c_int * n)()
    op = (ctypes.c_void_p * n)()
    ol = (ctypes.c_int * n)()
    be = (ctypes.c_int * n)(*[int(b) for b in backends])
    hp = (ctypes.c_void_p * n)(*[pl._h.value for pl in plans])
    for k in range(n):
        a, loc, kk = _vbuf(volts[k], getattr(plans[k], "in_type", None))
        vp[k], vl[k] = a, loc
        keep.append(kk)
        dt = np.complex64 if int(backends[k]) == 0 else np.float32
        b, loc2, kk2 = _buf(outs[k], dt, "out")
        op[k], ol[k] = b, loc2
        keep.append(kk2)
    _check(load().chirp_batch_run(hp, vp, vl, op, ol, be, n))


def chirp_combine_channels(P, first, last, f_c, bw: float, dump_len: int, dms, E,
                           k_dm: float = 0.0, stream=None) -> None:
    """Coarse channels aligned to the top channel and added (chirp_combine_channels).
    P: list of C contiguous float32 CUDA tensors [n_dm, n_dump, n_pix]; first,
    last: [C, n_dm] valid-dump bounds per channel; f_c: [C] centres (Hz);
    E: float32 CUDA tensor of P's shape."""
    import torch
    C = len(P)
    for t in list(P) + [E]:
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous() and t.shape == P[0].shape):
            raise TypeError("P and E must be contiguous float32 CUDA tensors of one shape")
    n_dm, n_dump, n_pix = P[0].shape
    fl = np.ascontiguousarray(np.asarray(first, np.int64).reshape(C, n_dm))
    la = np.ascontiguousarray(np.asarray(last, np.int64).reshape(C, n_dm))
    fc = np.ascontiguousarray(np.asarray(f_c, np.float64).ravel())
    dd = np.ascontiguousarray(np.asarray(dms, np.float64).ravel())
    if fc.size != C or dd.size != n_dm:
        raise ValueError("f_c must have one entry per channel and dms one per DM")
    ptrs = (ctypes.c_void_p * C)(*[t.data_ptr() for t in P])
    llp = ctypes.POINTER(ctypes.c_longlong)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(load().chirp_combine_channels(ptrs, C, int(n_dm), int(n_dump), int(n_pix),
                                         fl.ctypes.data_as(llp), la.ctypes.data_as(llp),
                                         fc.ctypes.data_as(dp), float(bw), int(dump_len),
                                         float(k_dm), dd.ctypes.data_as(dp),
                                         ctypes.c_void_p(E.data_ptr()), _stream_handle(stream)))


def chirp_last_error() -> str:
    return load().chirp_last_error().decode(errors="replace")


# ------------------------------------------------------------ convenience
class Plan:
    """Owns one chirp_plan (device workspace sized for one search shape)."""

    def __init__(self, xyz, f0: float, bw: float, n_samp: int, dms, dump_len: int,
                 nfft_min: int, pix_lm=None, k_dm: float = K_DM_DEFAULT,
                 beam_mode: int = BEAM_AUTO, n_ant: int | None = None, stream=None,
                 fb_chan: int = 0, fb_int: int = 1, fb_dm=None, flags: int = 0, fft_row: int = 0,
                 in_type: int = IN_C64, in_scale=None, beam_shape: int = 0,
                 corr_mode: int = CORR_AUTO):
        self._xyz = None if xyz is None else np.ascontiguousarray(xyz, dtype=np.float64)
        self._dms = np.ascontiguousarray(np.atleast_1d(dms), dtype=np.float64)
        self._pix = None if pix_lm is None else np.ascontiguousarray(pix_lm, dtype=np.float64)
        if n_ant is None:
            n_ant = int(self._xyz.shape[0])
        dp = ctypes.POINTER(ctypes.c_double)
        cfg = _Config()
        cfg.n_ant = int(n_ant)
        cfg.xyz_m = self._xyz.ctypes.data_as(dp) if self._xyz is not None else None
        cfg.f0_hz, cfg.bw_hz, cfg.k_dm = float(f0), float(bw), float(k_dm)
        cfg.n_samp = int(n_samp)
        cfg.dm = self._dms.ctypes.data_as(dp)
        cfg.n_dm = int(self._dms.size)
        cfg.dump_len = int(dump_len)
        cfg.nfft_min = int(nfft_min)
        cfg.pix_lm = self._pix.ctypes.data_as(dp) if self._pix is not None else None
        cfg.n_pix = 0 if self._pix is None else int(self._pix.shape[0])
        cfg.beam_mode = int(beam_mode)
        self._fb_dm = (None if fb_dm is None
                       else np.ascontiguousarray(np.atleast_1d(fb_dm), dtype=np.float64))
        cfg.fb_chan = int(fb_chan)
        cfg.fb_int = int(fb_int)
        cfg.fb_dm = self._fb_dm.ctypes.data_as(dp) if self._fb_dm is not None else None
        cfg.fb_n_dm = 0 if self._fb_dm is None else int(self._fb_dm.size)
        cfg.flags = int(flags)
        cfg.fft_row = int(fft_row)
        cfg.in_type = int(in_type)
        cfg.beam_shape = int(beam_shape)
        cfg.corr_mode = int(corr_mode)
        self.in_type = int(in_type)
        self._scale = (None if in_scale is None
                       else np.ascontiguousarray(np.atleast_1d(in_scale), dtype=np.float32))
        cfg.in_scale = (self._scale.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
                        if self._scale is not None else None)
        self.n_ant, self.n_samp, self.n_dm = cfg.n_ant, cfg.n_samp, cfg.n_dm
        self.n_pix = cfg.n_pix
        self._h = chirp_plan_create(cfg, stream)
        info = _Info()
        _check(load().chirp_plan_query(self._h, ctypes.byref(info)))
        self.n_dump = int(info.n_dump)
        self.n_pair = int(info.n_pair)
        self.info = {k: int(getattr(info, k)) for k, _ in _Info._fields_}

    @classmethod
    def from_scenario(cls, sc, **kw):
        return cls(sc.xyz, sc.f0, sc.bw, sc.n_samp, sc.dms, sc.dump_len, sc.nfft_min,
                   pix_lm=sc.pix_lm, k_dm=sc.k_dm, **kw)

    def close(self):
        if getattr(self, "_h", None):
            chirp_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def fft_split(self):
        """[(nfft, n_col, n_row)] of every FFT-length group (chirp_plan_fft_split)."""
        n = self.info["n_group"]
        nf = (ctypes.c_longlong * n)()
        nc = (ctypes.c_int * n)()
        nr = (ctypes.c_int * n)()
        _check(load().chirp_plan_fft_split(self._h, nf, nc, nr))
        return [(int(nf[g]), int(nc[g]), int(nr[g])) for g in range(n)]

    def dm_layout(self, d: int) -> dict:
        out = (ctypes.c_longlong * 7)()
        _check(load().chirp_dm_layout(self._h, int(d), out))
        keys = ("nfft", "n_hi", "n_lo", "n_hi_max", "n_lo_max", "step", "n_blk")
        return {k: int(v) for k, v in zip(keys, out)}

    def dump_range(self):
        first = (ctypes.c_longlong * self.n_dm)()
        last = (ctypes.c_longlong * self.n_dm)()
        _check(load().chirp_dump_range(self._h, first, last))
        return np.array(first[:], dtype=np.int64), np.array(last[:], dtype=np.int64)

    def dedisperse(self, volt, d: int, y_out):
        chirp_dedisperse_run(self._h, volt, d, y_out, self.in_type)
        return y_out

    def chirpolator(self, volt, vis_out):
        chirpolator_run(self._h, volt, vis_out, self.in_type)
        return vis_out

    def chimageator(self, volt, pow_out):
        chimageator_run(self._h, volt, pow_out, self.in_type)
        return pow_out

    def truedelay(self, volt, pow_out):
        """True-delay (wideband) beam powers [n_dm, n_dump, n_pix] (chirp_truedelay_run)."""
        vp, vl, _k1 = _vbuf(volt, self.in_type)
        op, ol, _k2 = _buf(pow_out, np.float32, "pow_out")
        _check(load().chirp_truedelay_run(self._h, vp, vl, op, ol))
        return pow_out

    def _mask(self, cell_mask):
        m = np.ascontiguousarray(cell_mask, dtype=np.uint8)
        if m.shape != (self.n_dm, self.n_dump):
            raise ValueError("cell_mask must be [n_dm, n_dump]")
        return m

    def chirpolator_selective(self, volt, cell_mask, vis_out):
        m = self._mask(cell_mask)
        vp, vl, _k1 = _vbuf(volt, self.in_type)
        op, ol, _k2 = _buf(vis_out, np.complex64, "vis_out")
        _check(load().chirpolator_run_selective(self._h, vp, vl, ctypes.c_void_p(m.ctypes.data),
                                                op, ol))
        return vis_out

    def chimageator_selective(self, volt, cell_mask, pow_out):
        m = self._mask(cell_mask)
        vp, vl, _k1 = _vbuf(volt, self.in_type)
        op, ol, _k2 = _buf(pow_out, np.float32, "pow_out")
        _check(load().chimageator_run_selective(self._h, vp, vl, ctypes.c_void_p(m.ctypes.data),
                                                op, ol))
        return pow_out

    def detect(self, pow_in, snr_min: float, max_cand: int = 1 << 16, with_stats: bool = False):
        """Candidates of dump powers [n_dm, n_dump, n_pix] (chirp_detect) as a
        numpy structured array (CANDIDATE_DTYPE) in (DM, dump, pixel) order;
        with_stats also returns the (median, sigma) array [n_dm, n_pix, 2]."""
        pp, pl, _k = _buf(pow_in, np.float32, "pow")
        out = np.zeros(max(int(max_cand), 0), dtype=CANDIDATE_DTYPE)
        st = np.zeros((self.n_dm, self.n_pix, 2), np.float32) if with_stats else None
        n = ctypes.c_longlong(0)
        _check(load().chirp_detect(self._h, pp, pl, float(snr_min),
                                   ctypes.c_void_p(out.ctypes.data) if out.size else None,
                                   int(out.size), CHIRP_HOST, ctypes.byref(n),
                                   ctypes.c_void_p(st.ctypes.data) if st is not None else None))
        if n.value > out.size:
            raise ChirpError(-2, "%d candidates exceed max_cand = %d" % (n.value, out.size))
        cands = out[:n.value].copy()
        return (cands, st) if with_stats else cands

    def status(self):
        """Raise ChirpError if a bounded device wait of an earlier run gave up."""
        _check(load().chirp_plan_status(self._h))

    def incoherent(self, volt, D_out, S_out=None):
        """Filterbank S [fb_chan, T_fb] (optional) and incoherent dedispersion
        D [fb_n_dm, T_fb] of the voltages (chirp_incoherent_run)."""
        vp, vl, _k1 = _vbuf(volt, self.in_type)
        dp_, dl, _k2 = _buf(D_out, np.float32, "D_out")
        sp_ = ctypes.c_void_p(0)
        if S_out is not None:
            sp_, sl, _k3 = _buf(S_out, np.float32, "S_out")
            if sl != dl:
                raise TypeError("S_out and D_out must live in the same place")
        _check(load().chirp_incoherent_run(self._h, vp, vl, sp_, dp_, dl))
        return D_out

    def stage_timing(self, enable, stages=None):
        """Per-stage device ms and launch counts since the last call; switches
        event timing on or off for later runs (synchronises the stream).
        stages: names from STAGES to time (None: every stage)."""
        ms = (ctypes.c_double * len(STAGES))()
        n = (ctypes.c_longlong * len(STAGES))()
        arg = int(bool(enable))
        if enable and stages is not None:
            arg = TIMING_SELECT
            for k in stages:
                arg |= 1 << STAGES.index(k)
        _check(load().chirp_stage_timing(self._h, arg, ms, n))
        return {k: (float(ms[j]), int(n[j])) for j, k in enumerate(STAGES)}


def _dev_f32(t, what):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
            and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % what)
    return ctypes.c_void_p(t.data_ptr())


class PropNet:
    """The learned proposer (chirp_propnet_*): 1-D conv net over the incoherent
    dedispersed power, trained and run by the library's kernels."""

    def __init__(self, n_dm: int, hidden: int, k1: int, k2: int, max_batch: int, n_time: int,
                 stream=None):
        self.n_dm, self.hidden, self.k1, self.k2 = n_dm, hidden, k1, k2
        self.max_batch, self.n_time = max_batch, n_time
        self._stream = _stream_handle(stream)
        h = ctypes.c_void_p()
        _check(load().chirp_propnet_create(ctypes.byref(h), n_dm, hidden, k1, k2, max_batch,
                                           n_time, self._stream))
        self._h = h
        self.n_params = int(load().chirp_propnet_param_count(h))

    def close(self):
        if getattr(self, "_h", None):
            load().chirp_propnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        a = np.ascontiguousarray(theta, dtype=np.float32)
        assert a.size == self.n_params
        _check(load().chirp_propnet_set_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def params(self) -> np.ndarray:
        a = np.empty(self.n_params, np.float32)
        _check(load().chirp_propnet_get_params(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return a

    def get_state(self) -> dict:
        """Parameters, Adam moments and Adam step (checkpoint of the trainer)."""
        arrs = [np.empty(self.n_params, np.float32) for _ in range(3)]
        step = ctypes.c_longlong(0)
        fpp = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in arrs]
        _check(load().chirp_propnet_get_state(self._h, *fpp, ctypes.byref(step)))
        return {"params": arrs[0], "m": arrs[1], "v": arrs[2], "step": int(step.value)}

    def set_state(self, state: dict) -> None:
        arrs = [np.ascontiguousarray(state[k], dtype=np.float32) for k in ("params", "m", "v")]
        for a in arrs:
            if a.size != self.n_params:
                raise ValueError("state arrays must hold %d values" % self.n_params)
        fpp = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in arrs]
        _check(load().chirp_propnet_set_state(self._h, *fpp, int(state["step"])))

    def grads(self) -> np.ndarray:
        a = np.empty(self.n_params, np.float32)
        _check(load().chirp_propnet_get_grads(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return a

    def forward(self, x, logits):
        _check(load().chirp_propnet_forward(self._h, _dev_f32(x, "x"), int(x.shape[0]),
                                            _dev_f32(logits, "logits")))
        return logits

    def backward(self, x, y, pos_weight: float) -> float:
        loss = ctypes.c_float()
        _check(load().chirp_propnet_backward(self._h, _dev_f32(x, "x"), _dev_f32(y, "y"),
                                             int(x.shape[0]), float(pos_weight), ctypes.byref(loss)))
        return float(loss.value)

    def train_step(self, x, y, pos_weight: float, lr: float) -> float:
        loss = ctypes.c_float()
        _check(load().chirp_propnet_train_step(self._h, _dev_f32(x, "x"), _dev_f32(y, "y"),
                                               int(x.shape[0]), float(pos_weight), float(lr),
                                               ctypes.byref(loss)))
        return float(loss.value)

    def normalize(self, D, x):
        _check(load().chirp_propnet_normalize(_dev_f32(D, "D"), int(D.shape[0]), int(D.shape[1]),
                                              _dev_f32(x, "x"), self._stream))
        return x

    def propose(self, logits, win: int, thr: float, mask):
        import torch
        assert mask.dtype == torch.int32 and mask.is_cuda
        _check(load().chirp_propose_windows(_dev_f32(logits, "logits"), int(logits.shape[0]),
                                            int(logits.shape[1]), int(win), float(thr),
                                            ctypes.c_void_p(mask.data_ptr()), self._stream))
        return mask
