"""Learned proposals for the coherent search: data, training and cell masks.

The pipeline (all numerical steps in the library's CUDA kernels):
  voltages --chirp_incoherent_run--> incoherent DM-time power D [n_dm, T_fb]
           --chirp_propnet_normalize--> per-DM z-scores x
           --chirp_propnet_forward--> logits z [n_dm, T_fb]
           --chirp_propose_windows--> proposal mask [n_dm, n_win]
           --cells()--> coherent (DM, dump) cell mask for *_run_selective.

The coherent plan and the incoherent grid share one DM list, so a proposed
window of DM d maps to the dumps covering that window (plus one window of
margin on each side).  Training segments come from the seeded sky model
(`skymodel`), with 0-4 dispersed bursts each (DM uniform, width log-uniform,
ideal-beam S/N uniform, direction a random beam centre) and a narrowband
interfering tone in 10 % of segments; labels mark the injected (DM, time)
cells.  Nothing here imports the oracle.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import Plan, PropNet, checkpoint, skymodel


@dataclasses.dataclass
class ProposalSetup:
    n_ant: int = 6
    max_baseline_m: float = 2000.0
    f0: float = 1.4e9
    bw: float = 8e6
    n_samp: int = 1 << 18
    dm_max: float = 150.0
    n_dm: int = 32
    nfft_min: int = 1 << 15
    dump_len: int = 1024
    n_side: int = 4
    field_deg: float = 1.0
    fb_chan: int = 32
    fb_int: int = 16
    win: int = 8              # filterbank samples per proposal window
    width_s: tuple = (20e-6, 1e-3)
    snr: tuple = (6.0, 30.0)
    max_pulses: int = 4
    rfi_frac: float = 0.1

    @property
    def dms(self) -> np.ndarray:
        return np.linspace(0.0, self.dm_max, self.n_dm)

    @property
    def t_fb(self) -> int:  # samples per filterbank sample
        return self.fb_chan * self.fb_int

    @property
    def T_fb(self) -> int:
        return self.n_samp // self.t_fb


def segment(setup: ProposalSetup, seed: int):
    """(voltages complex64 [M, N], list of Pulse) of one seeded training segment."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = skymodel.antenna_positions(setup.n_ant, setup.max_baseline_m, 4242)
    pix = skymodel.pixel_grid(setup.n_side, setup.field_deg)
    x = skymodel.noise(setup.n_ant, setup.n_samp, seed)
    pulses = []
    for i in range(int(rng.integers(0, setup.max_pulses + 1))):
        dm = float(rng.uniform(0.0, setup.dm_max))
        w = math.exp(rng.uniform(math.log(setup.width_s[0]), math.log(setup.width_s[1])))
        hi, lo = skymodel.sweep_samples(setup.f0, setup.bw, dm)
        guard = 8 * w * setup.bw + 64
        m_lo = int(math.ceil((hi + guard) / setup.dump_len))
        m_hi = int(math.floor((setup.n_samp - lo - guard) / setup.dump_len)) - 1
        if m_hi < m_lo:
            continue
        t0 = (int(rng.integers(m_lo, m_hi + 1)) + 0.5) * setup.dump_len
        snr = float(rng.uniform(*setup.snr))
        amp = skymodel.burst_amplitude(snr, setup.n_ant, setup.dump_len, w * setup.bw,
                                       setup.dump_len / 2)
        p = int(rng.integers(0, pix.shape[0]))
        pulse = skymodel.Pulse(dm, t0, w, amp, float(pix[p, 0]), float(pix[p, 1]),
                               seed * 16 + i + 1)
        skymodel.inject(x, xyz, setup.f0, setup.bw, pulse)
        pulses.append(pulse)
    if rng.random() < setup.rfi_frac:  # narrowband interference, common to all antennas
        f = rng.uniform(-0.45, 0.45) * setup.bw
        a = rng.uniform(0.3, 1.0)
        tone = (a * np.exp(2j * math.pi * f * np.arange(setup.n_samp) / setup.bw)).astype(np.complex64)
        x += tone[None, :]
    return x, pulses


def segment_device(setup: ProposalSetup, seed: int):
    """segment() drawn on the GPU: the same pulses (DM, time, width, S/N,
    direction, interference) for the same seed, with the noise and the bursts'
    own noise from torch's generator (skymodel.noise_device / inject_device).
    Returns (voltages complex64 CUDA tensor [M, N], list of Pulse)."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    xyz = skymodel.antenna_positions(setup.n_ant, setup.max_baseline_m, 4242)
    pix = skymodel.pixel_grid(setup.n_side, setup.field_deg)
    x = skymodel.noise_device(setup.n_ant, setup.n_samp, seed)
    pulses = []
    for i in range(int(rng.integers(0, setup.max_pulses + 1))):
        dm = float(rng.uniform(0.0, setup.dm_max))
        w = math.exp(rng.uniform(math.log(setup.width_s[0]), math.log(setup.width_s[1])))
        hi, lo = skymodel.sweep_samples(setup.f0, setup.bw, dm)
        guard = 8 * w * setup.bw + 64
        m_lo = int(math.ceil((hi + guard) / setup.dump_len))
        m_hi = int(math.floor((setup.n_samp - lo - guard) / setup.dump_len)) - 1
        if m_hi < m_lo:
            continue
        t0 = (int(rng.integers(m_lo, m_hi + 1)) + 0.5) * setup.dump_len
        snr = float(rng.uniform(*setup.snr))
        amp = skymodel.burst_amplitude(snr, setup.n_ant, setup.dump_len, w * setup.bw,
                                       setup.dump_len / 2)
        p = int(rng.integers(0, pix.shape[0]))
        pulse = skymodel.Pulse(dm, t0, w, amp, float(pix[p, 0]), float(pix[p, 1]),
                               seed * 16 + i + 1)
        skymodel.inject_device(x, xyz, setup.f0, setup.bw, pulse)
        pulses.append(pulse)
    if rng.random() < setup.rfi_frac:  # narrowband interference, common to all antennas
        f = rng.uniform(-0.45, 0.45) * setup.bw
        a = rng.uniform(0.3, 1.0)
        n = torch.arange(setup.n_samp, dtype=torch.float64, device=x.device)
        tone = (a * torch.exp(2j * math.pi * f * n / setup.bw)).to(torch.complex64)
        x += tone[None, :]
    return x, pulses


def _segment_job(args):
    setup, seed = args
    return segment(setup, seed)


def generate(setup: ProposalSetup, seeds, workers: int = 0):
    """Segments for the given seeds; a spawn-started process pool when workers > 0
    (start it before any CUDA work in the calling process)."""
    if workers <= 0:
        return [segment(setup, s) for s in seeds]
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_segment_job, [(setup, s) for s in seeds])


def labels(setup: ProposalSetup, pulses) -> np.ndarray:
    """y [n_dm, T_fb]: 1 at the nearest trial DM (and its neighbours) over the
    filterbank samples the burst covers at f0."""
    y = np.zeros((setup.n_dm, setup.T_fb), np.float32)
    ddm = setup.dms[1] - setup.dms[0] if setup.n_dm > 1 else 1.0
    for p in pulses:
        d = int(round(p.dm / ddm))
        half = max(1, int(math.ceil(0.5 * p.fwhm_s * setup.bw / setup.t_fb)))
        t = int(p.t0 // setup.t_fb)
        y[max(0, d - 1):d + 2, max(0, t - half):t + half + 1] = 1.0
    return y


class Proposer:
    """Incoherent features + the proposal network on one GPU."""

    def __init__(self, setup: ProposalSetup, hidden: int = 64, k1: int = 9, k2: int = 5,
                 max_batch: int = 16, seed: int = 7, stream=None):
        import torch
        self.s = setup
        self.torch = torch
        xyz = skymodel.antenna_positions(setup.n_ant, setup.max_baseline_m, 4242)
        self.plan = Plan(xyz, setup.f0, setup.bw, setup.n_samp, setup.dms, setup.dump_len,
                         setup.nfft_min, pix_lm=skymodel.pixel_grid(setup.n_side, setup.field_deg),
                         beam_mode=3, fb_chan=setup.fb_chan, fb_int=setup.fb_int,
                         fb_dm=setup.dms, stream=stream)
        self.net = PropNet(setup.n_dm, hidden, k1, k2, max_batch, setup.T_fb, stream=stream)
        rng = np.random.default_rng(seed)
        theta = []
        for shp in ((hidden, setup.n_dm, k1), (hidden,), (hidden, hidden, k2), (hidden,),
                    (setup.n_dm, hidden, 1), (setup.n_dm,)):
            if len(shp) == 3:
                theta.append(rng.standard_normal(shp) * math.sqrt(2.0 / (shp[1] * shp[2])))
            else:
                theta.append(np.zeros(shp))
        self.net.set_params(np.concatenate([t.ravel() for t in theta]).astype(np.float32))
        self._D = torch.empty((setup.n_dm, setup.T_fb), dtype=torch.float32, device="cuda")

    def features(self, x) -> "torch.Tensor":
        """Normalised incoherent DM-time power [n_dm, T_fb] on the device."""
        xd = x if isinstance(x, self.torch.Tensor) else self.torch.from_numpy(x).cuda()
        self.plan.incoherent(xd, self._D)
        out = self.torch.empty_like(self._D)
        self.net.normalize(self._D, out)
        return out

    def train(self, feats, ys, steps: int, batch: int, lr: float = 2e-3, pos_weight: float = 20.0,
              seed: int = 0, start_step: int = 0):
        """steps Adam steps on batches drawn from a generator seeded with seed;
        start_step > 0 resumes a trainer restored from a checkpoint taken
        after start_step steps (the batches it already drew are skipped, so
        the run continues exactly as the uninterrupted one)."""
        torch = self.torch
        X = torch.stack(feats)
        Y = torch.stack([torch.from_numpy(y) for y in ys]).cuda()
        g = np.random.default_rng(seed)
        for _ in range(start_step):
            g.choice(len(feats), size=batch, replace=False)
        losses = []
        for _ in range(steps):
            idx = torch.from_numpy(g.choice(len(feats), size=batch, replace=False)).cuda()
            losses.append(self.net.train_step(X[idx].contiguous(), Y[idx].contiguous(),
                                              pos_weight, lr))
        return losses

    def save(self, path: str) -> None:
        """Checkpoint of the trainer (network parameters, Adam state and step)."""
        checkpoint.save(self.net, path)

    def load(self, path: str) -> int:
        """Restore a checkpoint; returns the step to pass as start_step."""
        return checkpoint.load(self.net, path)

    def logits(self, feat) -> "torch.Tensor":
        z = self.torch.empty((1,) + tuple(feat.shape), dtype=self.torch.float32, device="cuda")
        self.net.forward(feat[None].contiguous(), z)
        return z[0]

    def propose(self, feat, thr: float) -> np.ndarray:
        """Proposal mask [n_dm, n_win] (numpy uint8)."""
        z = self.logits(feat)
        n_win = (self.s.T_fb + self.s.win - 1) // self.s.win
        m = self.torch.empty((self.s.n_dm, n_win), dtype=self.torch.int32, device="cuda")
        self.net.propose(z.contiguous(), self.s.win, thr, m)
        return m.cpu().numpy().astype(np.uint8)

    def cells(self, mask: np.ndarray, dm_margin: int = 1) -> np.ndarray:
        """Coherent (DM, dump) cell mask [n_dm, n_dump] of a proposal mask, with
        one window of margin in time and dm_margin trial DMs on each side (a
        burst between two trial DMs is detected on either)."""
        s = self.s
        return cells_of(mask, s.n_samp, s.dump_len, s.win * s.t_fb, dm_margin)


def cells_of(mask: np.ndarray, n_samp: int, dump_len: int, span: int,
             dm_margin: int = 1) -> np.ndarray:
    """Proposer.cells for any series length: mask [n_dm, n_win] of windows of
    span samples -> coherent cells [n_dm, n_samp // dump_len]."""
    n_dm = mask.shape[0]
    cells = np.zeros((n_dm, n_samp // dump_len), np.uint8)
    for d, w in zip(*np.nonzero(mask)):
        t_lo = max(0, (int(w) - 1) * span)
        t_hi = min(n_samp, (int(w) + 2) * span)
        d0, d1 = max(0, int(d) - dm_margin), min(n_dm, int(d) + dm_margin + 1)
        cells[d0:d1, t_lo // dump_len:(t_hi + dump_len - 1) // dump_len] = 1
    return cells


def recall(pulses_dets, cells_list, ddm: float, dump_len: int):
    """(found, total): of the injected pulses the full grid detects (a
    candidate within one trial DM and two dumps of the pulse), those with at
    least one such candidate inside the selected cells.  pulses_dets: per
    segment (pulses, set of (dm index, dump) candidates)."""
    found = tot = 0
    for (pulses, dets), cells in zip(pulses_dets, cells_list):
        for p in pulses:
            d = int(round(p.dm / ddm))
            m = int(p.t0 // dump_len)
            near = [(dd, mm) for (dd, mm) in dets if abs(dd - d) <= 1 and abs(mm - m) <= 2]
            if near:
                tot += 1
                found += any(cells[dd, mm] for dd, mm in near)
    return found, tot
