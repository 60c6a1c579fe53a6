"""CPU-only checks of the C-ABI library: it loads, exports every function the
public header declares, and rejects malformed plans in host code before any
CUDA call (no kernel runs here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1109_3186_gb300 as chirp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.isupper()))


def test_library_builds_and_exports_every_declared_symbol():
    lib = chirp.load()
    declared = _declared_functions()
    assert len(declared) >= 9
    for name in declared:
        assert hasattr(lib, name), name
    assert set(chirp.EXPORTED_SYMBOLS) <= set(declared)


def _cfg(**over):
    xyz = np.zeros((2, 3))
    dms = np.array([0.0, 10.0])
    base = dict(xyz=xyz, f0=1.4e9, bw=8e6, n_samp=1 << 14, dms=dms, dump_len=256,
                nfft_min=1 << 12)
    base.update(over)
    return base


@pytest.mark.parametrize("over,msg", [
    (dict(nfft_min=1000), "nfft_min"),
    (dict(nfft_min=128), "nfft_min"),
    (dict(dump_len=0), "dump_len"),
    (dict(dms=np.array([-1.0])), "negative"),
    (dict(bw=-1.0), "bw"),
    (dict(n_samp=0), "n_samp"),
    (dict(pix_lm=np.array([[0.9, 0.9]])), "l^2"),
    (dict(in_type=3), "in_type"),
    (dict(beam_mode=9), "beam_mode"),
    (dict(fft_row=300), "fft_row"),
    (dict(flags=8), "flag"),
    (dict(beam_shape=4), "beam_shape"),
    (dict(corr_mode=7), "corr_mode"),
    (dict(in_type=1, in_scale=np.array([np.inf, 1.0])), "in_scale"),
])
def test_plan_validation_rejects_bad_shapes(over, msg):
    with pytest.raises(chirp.ChirpError) as ei:
        chirp.Plan(**_cfg(**over))
    assert ei.value.code == -1
    assert msg in str(ei.value)


def test_graphs_flag_needs_a_stream():
    with pytest.raises(chirp.ChirpError) as ei:
        chirp.Plan(**_cfg(flags=chirp.FLAG_GRAPHS), stream=0)
    assert ei.value.code == -1 and "stream" in str(ei.value)


def test_forced_beam_kernel_shape_that_does_not_fit_is_refused():
    # 84 antennas, split-BF16: the weights of one row tile and two voltage
    # tiles exceed shared memory with 128-sample tiles (only the TMEM shape fits)
    xyz = np.zeros((84, 3))
    xyz[:, 0] = np.arange(84.0)
    with pytest.raises(chirp.ChirpError) as ei:
        chirp.Plan(**_cfg(xyz=xyz, pix_lm=np.zeros((4, 2)), beam_mode=chirp.BEAM_TC_3XBF16,
                          beam_shape=1))
    assert ei.value.code == -5 and "does not fit" in str(ei.value)


def test_watchdog_selftest_rejects_a_poll_count_out_of_range():
    rc, ms = chirp.chirp_watchdog_selftest(0)
    assert rc == chirp.CHIRP_EINVAL
    rc, ms = chirp.chirp_watchdog_selftest((1 << 24) + 1)
    assert rc == chirp.CHIRP_EINVAL


def _cpi(**over):
    from paper_1109_3186_gb300.cpi import CpiPlan
    base = dict(xyz=np.array([[0.0, 0, 0], [1000.0, 0, 0], [0, 800.0, 0]]), f0=1.4e9, bw=8e6,
                n_samp=1 << 14, dms=np.array([5.0, 10.0]), blk_len=256,
                pix_lm=np.array([[0.0, 0.0], [0.005, 0.0]]), half_width=2, max_bin=0)
    base.update(over)
    return CpiPlan(**base)


@pytest.mark.parametrize("over,msg", [
    (dict(xyz=np.zeros((1, 3))), "n_ant"),
    (dict(blk_len=100), "blk_len"),
    (dict(blk_len=8), "blk_len"),
    (dict(n_samp=100), "n_samp"),
    (dict(dms=np.array([0.0])), "DM"),
    (dict(dms=np.array([5000.0])), "longer than the data"),
    (dict(half_width=9), "half_width"),
    (dict(max_bin=65), "max_bin"),
    (dict(max_bin=1), "below"),
    (dict(bw=0.0), "bw_hz"),
    (dict(pix_lm=np.array([[0.9, 0.9]])), "l^2"),
])
def test_cpi_plan_validation_rejects_bad_shapes(over, msg):
    with pytest.raises(chirp.ChirpError) as ei:
        _cpi(**over)
    assert ei.value.code == -1
    assert msg in str(ei.value)


@pytest.mark.parametrize("over,msg", [
    (dict(n_ant=1), "n_ant"),
    (dict(n_ant=40), "n_ant"),
    (dict(spacing_m=0.0), "spacing_m"),
    (dict(n_spatial=4), "n_spatial"),
    (dict(half_width=5, n_spatial=8), "half_width"),
    (dict(dms=[0.0]), "DM"),
    (dict(dms=[5000.0]), "longer than the data"),
    (dict(dump_len=0), "dump_len"),
    (dict(l_dir=[0.0, 1.5]), "l_dir"),
])
def test_chimg_plan_validation_rejects_bad_shapes(over, msg):
    from paper_1109_3186_gb300.chimg import ChimgPlan
    base = dict(n_ant=6, spacing_m=50.0, f0=1.4e9, bw=8e6, n_samp=1 << 14, dms=[5.0], dump_len=256,
                l_dir=[0.0, 0.01], n_spatial=16, half_width=1)
    base.update(over)
    with pytest.raises(chirp.ChirpError) as ei:
        ChimgPlan(**base)
    assert ei.value.code == -1
    assert msg in str(ei.value)
