"""The device variants of the sky model follow the host model: inject_device
with the host's burst noise reproduces inject() (run here on torch's CPU
device), and noise_device has the host noise model's moments."""
import math

import numpy as np
import pytest

from paper_1109_3186_gb300 import skymodel

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dm,l,m", [(0.0, 0.0, 0.0), (37.5, 0.004, -0.002), (140.0, -0.006, 0.001)])
def test_inject_device_equals_inject_with_the_same_burst_noise(dm, l, m):
    n_ant, n_samp, f0, bw = 5, 1 << 16, 1.4e9, 8e6
    xyz = skymodel.antenna_positions(n_ant, 2000.0, 3)
    p = skymodel.Pulse(dm, 30000.5, 200e-6, 0.7, l, m, 99)
    x = np.zeros((n_ant, n_samp), np.complex64)
    skymodel.inject(x, xyz, f0, bw, p)
    # the same window and burst noise as inject() draws
    w = p.fwhm_s * bw
    hi, lo = skymodel.sweep_samples(f0, bw, dm)
    gmax = float(np.max(np.abs(skymodel.geometric_delay(xyz, l, m)))) * bw
    margin = int(math.ceil(6.0 * w + gmax + 64))
    nfft = 1 << int(math.ceil(math.log2(int(math.ceil(hi + lo)) + 2 * margin)))
    rng = np.random.Generator(np.random.PCG64(p.seed))
    ns = (rng.standard_normal(nfft) + 1j * rng.standard_normal(nfft)) / math.sqrt(2.0)
    xt = torch.zeros((n_ant, n_samp), dtype=torch.complex64)
    skymodel.inject_device(xt, xyz, f0, bw, p, burst_noise=torch.from_numpy(ns))
    assert np.abs(x).max() > 0.1
    assert np.max(np.abs(xt.numpy() - x)) < 1e-6 * np.abs(x).max()


def test_noise_device_moments():
    z = skymodel.noise_device(3, 1 << 16, 11, device="cpu").numpy()
    assert z.dtype == np.complex64
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.02
    assert abs(np.mean(z.real ** 2) - 0.5) < 0.02 and abs(np.mean(z.real * z.imag)) < 0.01
    assert not np.array_equal(z, skymodel.noise_device(3, 1 << 16, 12, device="cpu").numpy())
    assert np.array_equal(z, skymodel.noise_device(3, 1 << 16, 11, device="cpu").numpy())
