"""Seeded synthetic antenna voltages: the sky model that feeds the pulse search.

This module produces INPUTS only.  It models what an array of antennas records
when a dispersed radio pulse arrives from some direction on top of receiver
noise; it holds no step of the search itself (no dedispersion, no correlation,
no beamforming).  Both the FP64 oracle and the CUDA path consume what it makes,
and neither of them imports anything else from the other.

Physical model (all FP64 on the host, numpy only):

* Receiver noise: per antenna, independent unit-variance circular complex
  Gaussian samples, E|n|^2 = 1 (each component sigma = 1/sqrt(2)).
* Pulse: an amplitude-modulated noise burst a * sqrt(g(t - t0)) * n_s(t) common
  to all antennas, g a Gaussian of full width at half maximum W and unit peak.
  Real pulsar/FRB emission is such a burst; its spectrum fills the whole band,
  which is what dispersion then smears.
* Cold-plasma dispersion (Sec. 2.1, Eq. 1): a component at radio frequency nu
  arrives k*DM/nu^2 later than at infinite frequency.  Integrating that delay
  over frequency gives the propagation phase 2*pi*k*DM/nu; with nu = f0 + f
  and the constant and the bulk delay at f0 removed, the phase applied to the
  baseband spectrum is  2*pi*k*DM*(1/(f0+f) - 1/f0 + f/f0^2).  Time stamps
  therefore refer to the arrival at the band centre f0.
* Geometry (App. A.1, Eq. tau3D): antenna a records the wavefront
  tau_a = (x l + y m + z (sqrt(1 - l^2 - m^2) - 1)) / c  later than the array
  origin; the whole RF phase exp(-2 pi j (f0 + f) tau_a) is applied.

All draws come from numpy's PCG64 with explicit seeds, so every input is
reproducible bit for bit on any host.  The device variants at the end
(noise_device, inject_device) apply the same model to a torch tensor on the
GPU, with torch's seeded generator for the noise draws: they serve bulk
training data, where moving each segment from host worker processes would
dominate, and they are not equal sample for sample to the host versions.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

C_LIGHT = 299792458.0          # m/s (exact, SI definition)
K_DM = 4.148808e15             # s Hz^2 / (pc cm^-3); Sec. 2.1 gives 4.15 ms GHz^2


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------
def antenna_positions(n_ant: int, max_baseline_m: float, seed: int) -> np.ndarray:
    """Uniform-random positions in a disc of diameter ``max_baseline_m`` (z = 0).

    Returns float64 [n_ant, 3] metres in the (u, v, w) frame, w towards the
    phase centre.  Any two antennas are therefore at most max_baseline_m apart.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    r = 0.5 * max_baseline_m * np.sqrt(rng.random(n_ant))
    phi = 2.0 * math.pi * rng.random(n_ant)
    xyz = np.zeros((n_ant, 3), dtype=np.float64)
    xyz[:, 0] = r * np.cos(phi)
    xyz[:, 1] = r * np.sin(phi)
    return xyz


def pixel_grid(n_side: int, field_deg: float) -> np.ndarray:
    """Direction cosines (l, m) of an n_side x n_side grid of beam centres.

    The grid spans a square of ``field_deg`` on a side centred on boresight;
    pixel (i, j) sits at angle ((i + 1/2) * delta - field/2) in each axis and
    l = sin(angle_x), m = sin(angle_y).  Row-major: pixel index = j*n_side + i.
    Returns float64 [n_side*n_side, 2].
    """
    delta = math.radians(field_deg) / n_side
    ang = (np.arange(n_side) + 0.5) * delta - 0.5 * math.radians(field_deg)
    ax, ay = np.meshgrid(np.sin(ang), np.sin(ang), indexing="xy")
    return np.stack([ax.ravel(), ay.ravel()], axis=1).astype(np.float64)


def geometric_delay(xyz: np.ndarray, l: float, m: float) -> np.ndarray:
    """Per-antenna wavefront delay in seconds for direction (l, m) (Eq. tau3D)."""
    n = math.sqrt(max(0.0, 1.0 - l * l - m * m))
    return (xyz[:, 0] * l + xyz[:, 1] * m + xyz[:, 2] * (n - 1.0)) / C_LIGHT


def sweep_samples(f0: float, bw: float, dm: float, k_dm: float = K_DM) -> tuple[float, float]:
    """Dispersion sweep (samples) above and below f0 over the band, Eq. 1."""
    hi = k_dm * dm * (1.0 / f0 ** 2 - 1.0 / (f0 + bw / 2) ** 2) * bw
    lo = k_dm * dm * (1.0 / (f0 - bw / 2) ** 2 - 1.0 / f0 ** 2) * bw
    return hi, lo


# --------------------------------------------------------------------------
# signals
# --------------------------------------------------------------------------
def noise(n_ant: int, n_samp: int, seed: int) -> np.ndarray:
    """Unit-variance circular complex Gaussian noise, complex64 [n_ant, n_samp]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = np.empty((n_ant, n_samp), dtype=np.complex64)
    s = np.float32(1.0 / math.sqrt(2.0))
    for a in range(n_ant):  # per antenna keeps the peak host memory small
        re = rng.standard_normal(n_samp, dtype=np.float32)
        im = rng.standard_normal(n_samp, dtype=np.float32)
        out[a].real = re * s
        out[a].imag = im * s
    return out


@dataclasses.dataclass
class Pulse:
    dm: float            # pc cm^-3
    t0: float            # arrival time at f0, in samples
    fwhm_s: float        # Gaussian FWHM of the intensity envelope, seconds
    amp: float           # peak voltage amplitude a (noise rms is 1)
    l: float             # direction cosines of the source
    m: float
    seed: int            # seed of the burst's own noise


def burst_amplitude(snr: float, n_ant: int, dump_len: int, fwhm_samp: float,
                    offset_in_dump: float) -> float:
    """Amplitude a giving the ideal beam dump-integrated S/N ``snr``.

    For the coherent sum of M antennas at the true DM and direction, the noise
    power per sample is exponential with mean M and standard deviation M, so a
    dump of L samples has noise std M*sqrt(L); the pulse adds M^2 a^2 sum g.
    Hence S/N = M a^2 (sum over the dump of g) / sqrt(L).
    """
    t = np.arange(dump_len) - offset_in_dump
    g = np.exp(-4.0 * math.log(2.0) * (t / fwhm_samp) ** 2)
    return math.sqrt(snr * math.sqrt(dump_len) / (n_ant * float(g.sum())))


def inject(x: np.ndarray, xyz: np.ndarray, f0: float, bw: float, p: Pulse,
           k_dm: float = K_DM) -> None:
    """Add one dispersed, geometrically delayed burst to x [n_ant, n_samp] in place."""
    n_ant, n_samp = x.shape
    w = p.fwhm_s * bw                                  # FWHM in samples
    hi, lo = sweep_samples(f0, bw, p.dm, k_dm)
    tau = geometric_delay(xyz, p.l, p.m)
    gmax = float(np.max(np.abs(tau))) * bw
    margin = int(math.ceil(6.0 * w + gmax + 64))
    start = int(math.floor(p.t0 - hi)) - margin
    length = int(math.ceil(hi + lo)) + 2 * margin
    nfft = 1 << int(math.ceil(math.log2(length)))
    # undispersed burst on the window grid
    rng = np.random.Generator(np.random.PCG64(p.seed))
    t = np.arange(nfft, dtype=np.float64) + start - p.t0
    env = np.exp(-2.0 * math.log(2.0) * (t / w) ** 2)   # sqrt of the intensity Gaussian
    env[np.abs(t) > 8.0 * w] = 0.0
    ns = (rng.standard_normal(nfft) + 1j * rng.standard_normal(nfft)) / math.sqrt(2.0)
    burst = p.amp * env * ns
    spec = np.fft.fft(burst)
    f = np.fft.fftfreq(nfft, d=1.0 / bw)
    disp = 2.0 * math.pi * k_dm * p.dm * (1.0 / (f0 + f) - 1.0 / f0 + f / f0 ** 2)
    spec = spec * np.exp(1j * disp)
    lo_i, hi_i = max(start, 0), min(start + nfft, n_samp)
    if hi_i <= lo_i:
        return
    for a in range(n_ant):
        sa = spec * np.exp(-2j * math.pi * (f0 + f) * tau[a])
        sig = np.fft.ifft(sa)
        x[a, lo_i:hi_i] += sig[lo_i - start:hi_i - start].astype(np.complex64)


# --------------------------------------------------------------------------
# the array scenarios
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Scenario:
    name: str
    xyz: np.ndarray                 # [M, 3] float64
    f0: float
    bw: float
    n_samp: int
    dms: np.ndarray                 # [n_dm] float64
    dump_len: int
    nfft_min: int
    pix_lm: np.ndarray | None       # [n_pix, 2] float64, or None
    pulses: list
    seed: int
    k_dm: float = K_DM

    @property
    def n_ant(self) -> int:
        return int(self.xyz.shape[0])

    def voltages(self) -> np.ndarray:
        x = noise(self.n_ant, self.n_samp, self.seed)
        for p in self.pulses:
            inject(x, self.xyz, self.f0, self.bw, p, self.k_dm)
        return x


def _place_pulse(rng, dm, f0, bw, n_samp, dump_len, k_dm, guard):
    hi, lo = sweep_samples(f0, bw, dm, k_dm)
    m_lo = int(math.ceil((hi + guard) / dump_len))
    m_hi = int(math.floor((n_samp - lo - guard) / dump_len)) - 1
    if m_hi < m_lo:
        return None
    m = int(rng.integers(m_lo, m_hi + 1))
    return (m + 0.5) * dump_len


def chirpolator_small(n_samp: int = 1 << 20, n_dm: int = 16, seed: int = 1001,
                      n_ant: int = 6, dm_max: float = 150.0, nfft_min: int = 1 << 16,
                      dump_len: int = 1024, bw: float = 8e6, f0: float = 1.4e9,
                      with_pulse: bool = True) -> Scenario:
    """6 antennas within 2 km, 8 MHz at 1.4 GHz, 16 DMs in 0-150, FFT 2^16, dump 1024.

    One burst: DM 75, 50 us FWHM, ideal-beam S/N 20, 0.5 deg off boresight.
    Sizes can be shrunk for the oracle's quick checks.
    """
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    xyz = antenna_positions(n_ant, 2000.0, seed)
    dms = np.linspace(0.0, dm_max, n_dm)
    pulses = []
    if with_pulse:
        dm_p = 0.5 * dm_max
        fw = 50e-6
        guard = 8 * fw * bw + 64
        t0 = _place_pulse(rng, dm_p, f0, bw, n_samp, dump_len, K_DM, guard)
        if t0 is not None:
            phi = 2 * math.pi * rng.random()
            th = math.radians(0.5)
            amp = burst_amplitude(20.0, n_ant, dump_len, fw * bw, dump_len / 2)
            pulses.append(Pulse(dm_p, t0, fw, amp, math.sin(th) * math.cos(phi),
                                math.sin(th) * math.sin(phi), seed + 11))
    return Scenario("chirpolator 6 ant, 8 MHz, 2^%d samples, %d DMs" % (int(math.log2(n_samp)), n_dm),
                    xyz, f0, bw, n_samp, dms, dump_len, nfft_min, None, pulses, seed)


def chimageator_medium(n_samp: int = 1 << 22, n_dm: int = 64, seed: int = 1002,
                       n_ant: int = 12, dm_max: float = 300.0, nfft_min: int = 1 << 18,
                       dump_len: int = 4096, bw: float = 32e6, f0: float = 1.4e9,
                       n_side: int = 32, field_deg: float = 1.0, n_pulse: int = 3) -> Scenario:
    """12 antennas within 6 km, 32 MHz at 1.4 GHz, 64 DMs in 0-300, FFT >= 2^18,
    32x32 beams over 1 deg, dump 4096; 3 bursts at seeded DM, time and pixel
    (50 us FWHM, ideal-beam S/N 20 each)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    xyz = antenna_positions(n_ant, 6000.0, seed)
    dms = np.linspace(0.0, dm_max, n_dm)
    pix = pixel_grid(n_side, field_deg)
    pulses = []
    fw = 50e-6
    for i in range(n_pulse):
        dm_p = float(rng.uniform(0.0, dm_max))
        guard = 8 * fw * bw + 64
        t0 = _place_pulse(rng, dm_p, f0, bw, n_samp, dump_len, K_DM, guard)
        if t0 is None:
            continue
        pidx = int(rng.integers(0, pix.shape[0]))
        amp = burst_amplitude(20.0, n_ant, dump_len, fw * bw, dump_len / 2)
        pulses.append(Pulse(dm_p, t0, fw, amp, float(pix[pidx, 0]), float(pix[pidx, 1]),
                            seed + 100 + i))
    return Scenario("chimageator 12 ant, 32 MHz, 2^%d samples, %d DMs, %d beams"
                    % (int(math.log2(n_samp)), n_dm, pix.shape[0]),
                    xyz, f0, bw, n_samp, dms, dump_len, nfft_min, pix, pulses, seed)


# --------------------------------------------------------------------------
# int8 voltages (the precision form's ingest format)
# --------------------------------------------------------------------------
def quantize_ci8(x: np.ndarray, counts_rms: float = 16.0):
    """Complex int8 voltages as a digitiser would record them.

    Per antenna the gain puts the per-component RMS at ``counts_rms`` counts;
    each component is rounded half to even and clamped to +-127.  Returns
    (q int8 [M, N, 2] interleaved (re, im), scale float32 [M]) with
    x ~= scale[a] * (q[a, :, 0] + j q[a, :, 1]).
    """
    M = x.shape[0]
    q = np.empty((M, x.shape[1], 2), np.int8)
    scale = np.empty(M, np.float32)
    for a in range(M):
        rms = math.sqrt(float(np.mean(np.abs(x[a].astype(np.complex128)) ** 2)) / 2.0)
        g = counts_rms / rms if rms > 0 else 1.0
        scale[a] = np.float32(1.0 / g)
        q[a, :, 0] = np.clip(np.rint(x[a].real * g), -127, 127)
        q[a, :, 1] = np.clip(np.rint(x[a].imag * g), -127, 127)
    return q, scale


def dequantize_ci8(q: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """complex64 [M, N]: scale[a] * (re + j im), each product rounded to FP32
    (what the int8 ingest computes before the first FFT pass)."""
    s = scale.astype(np.float32)[:, None]
    re = q[..., 0].astype(np.float32) * s
    im = q[..., 1].astype(np.float32) * s
    return (re + 1j * im).astype(np.complex64)


def precision_form(channel: int = 0, n_chan: int = 8, n_samp: int = 1 << 24, n_dm: int = 256,
                   dm_min: float = 1.0, dm_max: float = 2000.0, seed: int = 1003,
                   n_ant: int = 36, n_side: int = 64, field_deg: float = 1.0,
                   dump_len: int = 4096, nfft_min: int = 1 << 16, chan_bw: float = 42e6,
                   f_centre: float = 1.4e9, n_pulse: int = 1) -> Scenario:
    """One coarse channel of the sparse 36-antenna array (6 km maximum
    baseline): 8 x 42 MHz channels around 1.4 GHz, channel c centred at
    f_centre + (c - (n_chan - 1) / 2) chan_bw; trial DMs 0 and then n_dm - 1
    log-spaced from dm_min to dm_max; 64 x 64 beams.  Voltages are meant to be quantised with
    quantize_ci8 before the search."""
    f0 = f_centre + (channel - 0.5 * (n_chan - 1)) * chan_bw
    rng = np.random.Generator(np.random.PCG64(seed + 7 + 1000 * channel))
    xyz = antenna_positions(n_ant, 6000.0, seed)
    dms = np.concatenate([[0.0], np.geomspace(dm_min, dm_max, n_dm - 1)])
    pix = pixel_grid(n_side, field_deg)
    pulses = []
    fw = 50e-6
    for i in range(n_pulse):
        dm_p = float(np.exp(rng.uniform(math.log(dm_min), math.log(dm_max))))
        guard = 8 * fw * chan_bw + 64
        t0 = _place_pulse(rng, dm_p, f0, chan_bw, n_samp, dump_len, K_DM, guard)
        if t0 is None:
            continue
        pidx = int(rng.integers(0, pix.shape[0]))
        amp = burst_amplitude(20.0, n_ant, dump_len, fw * chan_bw, dump_len / 2)
        pulses.append(Pulse(dm_p, t0, fw, amp, float(pix[pidx, 0]), float(pix[pidx, 1]),
                            seed + 100 + i + 1000 * channel))
    return Scenario("precision form: 36 ant, channel %d of %d x %.0f MHz, 2^%d samples, %d DMs"
                    % (channel, n_chan, chan_bw / 1e6, int(math.log2(n_samp)), n_dm),
                    xyz, f0, chan_bw, n_samp, dms, dump_len, nfft_min, pix, pulses,
                    seed + 1000 * channel)


# --------------------------------------------------------------------------
# dump-power fields (inputs of the candidate detection alone)
# --------------------------------------------------------------------------
def power_field(n_dm: int, n_dump: int, n_pix: int, first, last, seed: int,
                mean: float = 1.0, n_peaks: int = 0, peak_scale: float = 30.0) -> np.ndarray:
    """float32 [n_dm, n_dump, n_pix] of exponentially distributed dump powers
    (the chi-squared noise of a detected beam) inside each DM's valid dumps
    [first[d], last[d]], zero outside, plus n_peaks seeded bright cells of
    mean * (1 + peak_scale * U(0.5, 1))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    P = np.zeros((n_dm, n_dump, n_pix), np.float32)
    for d in range(n_dm):
        f, l = int(first[d]), int(last[d])
        if l >= f:
            P[d, f:l + 1] = (mean * rng.exponential(size=(l - f + 1, n_pix))).astype(np.float32)
    for _ in range(n_peaks):
        d = int(rng.integers(0, n_dm))
        f, l = int(first[d]), int(last[d])
        if l < f:
            continue
        m = int(rng.integers(f, l + 1))
        p = int(rng.integers(0, n_pix))
        P[d, m, p] = np.float32(mean * (1.0 + peak_scale * rng.uniform(0.5, 1.0)))
    return P


# --------------------------------------------------------------------------
# device variants (bulk training segments)
# --------------------------------------------------------------------------
def noise_device(n_ant: int, n_samp: int, seed: int, device="cuda"):
    """The noise model of noise() drawn on the device: complex64 tensor
    [n_ant, n_samp] from torch's generator seeded with ``seed``."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    re = torch.randn((n_ant, n_samp), generator=g, device=device, dtype=torch.float32)
    im = torch.randn((n_ant, n_samp), generator=g, device=device, dtype=torch.float32)
    return torch.complex(re, im) * (1.0 / math.sqrt(2.0))


def inject_device(x, xyz: np.ndarray, f0: float, bw: float, p: Pulse, k_dm: float = K_DM,
                  burst_noise=None) -> None:
    """inject() for a torch tensor x [n_ant, n_samp] (complex64), in place: the
    same window, envelope, dispersion phase and geometric delays in FP64 on
    x's device.  The burst's unit-variance noise is burst_noise (complex128
    [nfft], e.g. to reproduce inject() exactly) or drawn from torch's
    generator seeded with p.seed."""
    import torch
    dev = x.device
    n_ant, n_samp = x.shape
    w = p.fwhm_s * bw
    hi, lo = sweep_samples(f0, bw, p.dm, k_dm)
    tau = geometric_delay(xyz, p.l, p.m)
    gmax = float(np.max(np.abs(tau))) * bw
    margin = int(math.ceil(6.0 * w + gmax + 64))
    start = int(math.floor(p.t0 - hi)) - margin
    length = int(math.ceil(hi + lo)) + 2 * margin
    nfft = 1 << int(math.ceil(math.log2(length)))
    lo_i, hi_i = max(start, 0), min(start + nfft, n_samp)
    if hi_i <= lo_i:
        return
    t = torch.arange(nfft, dtype=torch.float64, device=dev) + float(start - p.t0)
    env = torch.exp(-2.0 * math.log(2.0) * (t / w) ** 2)
    env[torch.abs(t) > 8.0 * w] = 0.0
    if burst_noise is None:
        g = torch.Generator(device=dev)
        g.manual_seed(int(p.seed))
        burst_noise = torch.complex(
            torch.randn(nfft, generator=g, device=dev, dtype=torch.float64),
            torch.randn(nfft, generator=g, device=dev, dtype=torch.float64)) / math.sqrt(2.0)
    burst = p.amp * env * burst_noise.to(dev)
    spec = torch.fft.fft(burst)
    f = torch.fft.fftfreq(nfft, d=1.0 / bw, device=dev, dtype=torch.float64)
    disp = 2.0 * math.pi * k_dm * p.dm * (1.0 / (f0 + f) - 1.0 / f0 + f / f0 ** 2)
    spec = spec * torch.exp(1j * disp)
    for a in range(n_ant):
        sa = spec * torch.exp(-2j * math.pi * (f0 + f) * float(tau[a]))
        sig = torch.fft.ifft(sa)
        x[a, lo_i:hi_i] += sig[lo_i - start:hi_i - start].to(torch.complex64)
