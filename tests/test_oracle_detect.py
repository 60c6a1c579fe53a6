"""Pins of the oracle's candidate detection (median / 1.4826 MAD S/N per
(DM, pixel) series, local maxima over (DM, dump, pixel) +- 1):

- the series statistics against numpy's median, and against the normal
  distribution (1.4826 MAD estimates the standard deviation);
- hand-computed S/N of tiny series (odd and even lengths);
- the local-maximum rule against scipy.ndimage's maximum filter;
- invalid dumps take no part in the statistics or the neighbourhoods.
"""
import numpy as np
import pytest

import oracle as orc

ndimage = pytest.importorskip("scipy.ndimage")


def test_stats_match_numpy_median_odd_and_even():
    rng = np.random.default_rng(4)
    P = rng.exponential(size=(3, 41, 5)).astype(np.float32)
    first, last = np.array([0, 3, 1]), np.array([40, 38, 39])   # 41, 36, 39 values
    st = orc.series_stats(P, first, last)
    for d in range(3):
        for p in range(5):
            x = P[d, first[d]:last[d] + 1, p]
            med = np.median(x)
            assert st[d, p, 0] == med
            assert st[d, p, 1] == np.float32(1.4826) * np.median(np.abs(x - med))


def test_mad_estimates_gaussian_sigma():
    rng = np.random.default_rng(5)
    P = (3.0 + 2.0 * rng.standard_normal((1, 200001, 1))).astype(np.float32)
    st = orc.series_stats(P, [0], [200000])
    assert abs(st[0, 0, 0] - 3.0) < 0.02
    assert abs(st[0, 0, 1] - 2.0) < 0.03


@pytest.mark.parametrize("series,dump,snr", [
    ([1, 2, 3, 4, 100], 4, 97 / 1.4826),          # med 3, MAD 1
    ([1, 2, 3, 4, 5, 100], 5, 96.5 / (1.4826 * 1.5)),  # med 3.5, MAD 1.5
])
def test_hand_computed_snr(series, dump, snr):
    P = np.array(series, np.float32)[None, :, None]
    n = len(series)
    d, m, p, s = orc.detect(P, [0], [n - 1], 6.0)
    assert list(d) == [0] and list(m) == [dump] and list(p) == [0]
    assert s[0] == pytest.approx(snr, rel=1e-6)


def test_local_maxima_match_maximum_filter():
    rng = np.random.default_rng(6)
    n_dm, n_dump, n_pix = 5, 60, 9
    P = rng.exponential(size=(n_dm, n_dump, n_pix)).astype(np.float32)
    first = np.zeros(n_dm, np.int64)
    last = np.full(n_dm, n_dump - 1)
    thr = 2.0
    st = orc.series_stats(P, first, last)
    snr = (P - st[:, None, :, 0]) / st[:, None, :, 1]
    peak = snr == ndimage.maximum_filter(snr, size=3, mode="constant", cval=-np.inf)
    want = np.argwhere(peak & (snr >= thr))
    d, m, p, s = orc.detect(P, first, last, thr)
    got = np.stack([d, m, p], 1)
    assert len(want) > 20
    assert np.array_equal(got, want)
    assert np.allclose(s, snr[d, m, p], rtol=1e-6)


def test_invalid_dumps_are_outside_stats_and_neighbourhoods():
    rng = np.random.default_rng(7)
    P = rng.exponential(size=(2, 30, 3)).astype(np.float32)
    first, last = np.array([0, 10]), np.array([29, 19])
    P[1, :10] = 1e9                 # invalid dumps of DM 1: ignored everywhere
    P[1, 20:] = 1e9
    P[0, 25, 1] = 50.0              # peak of DM 0 next to DM 1's invalid dump 25
    st = orc.series_stats(P, first, last)
    ref = P[1, 10:20, 2]
    assert st[1, 2, 0] == np.median(ref)
    d, m, p, s = orc.detect(P, first, last, 6.0)
    assert (0, 25, 1) in set(zip(d.tolist(), m.tolist(), p.tolist()))
    assert np.all((m[d == 1] >= 10) & (m[d == 1] <= 19))
