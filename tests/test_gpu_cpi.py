"""Parity of the CUDA Chirpolator pre-integrator (chirp_cpi_*) with the FP64
oracle (oracle/cpi.py): partial DFTs V, window DFTs X and images E element by
element on small seeded cases (ragged tails, one to 276 pairs, F = 0 and
explicit K; the image both as the dense tensor-core contraction and as the
sparse CUDA-core gathers), device and host buffers, the bins each pair computes, a
dispersed burst from the sky model found at its pixel and DM, and sampled
windows of the 12-antenna, 2^22-sample, 63-DM workload.

Tolerances (FP32 arithmetic, unit roundoff u = 6e-8): a partial DFT sums L
mixed products, so its error is at most ~sqrt(L) u of the block's scale
(1e-6 at L = 256) plus the Taylor truncation (1e-9) and FP32 phases
(~3e-7 rad); the window DFTs add the blocks in compensated FP32 (two
floats per sum).  V and X are held to
2e-5 of their largest magnitude per DM, E = |P|^2 to 1e-4 of its largest
value per DM."""
import math

import numpy as np
import pytest

from oracle import cpi as ocpi
from paper_1109_3186_gb300 import skymodel
from paper_1109_3186_gb300.cpi import CpiPlan

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K_DM = skymodel.K_DM


def _case(n_ant, n_samp, dms, L, bw, field_deg, n_side, max_b, seed, F=2, max_bin=0, pulse=True):
    xyz = skymodel.antenna_positions(n_ant, max_b, seed)
    xyz[:, 2] = np.random.default_rng(seed).uniform(-15, 15, n_ant)
    pix = skymodel.pixel_grid(n_side, field_deg)
    x = skymodel.noise(n_ant, n_samp, seed + 1)
    if pulse:
        dm = float(dms[len(dms) // 2])
        p = skymodel.Pulse(dm=dm, t0=0.6 * n_samp, fwhm_s=20e-6, amp=2.0, l=pix[n_side + 1][0],
                           m=pix[n_side + 1][1], seed=seed + 2)
        skymodel.inject(x, xyz, 1.4e9, bw, p)
    return dict(xyz=xyz, f0=1.4e9, bw=bw, n_samp=n_samp, dms=np.asarray(dms, float), blk_len=L,
                pix_lm=pix, half_width=F, max_bin=max_bin), x


CASES = {
    "5ant_ragged": dict(n_ant=5, n_samp=(1 << 15) + 100, dms=[3.0, 12.0, 45.0, 150.0], L=256, bw=8e6,
                        field_deg=1.5, n_side=4, max_b=3000.0, seed=11),
    "3ant_F0_fixedK": dict(n_ant=3, n_samp=64 * 40 + 17, dms=[1.0, 2.5], L=64, bw=16e6, field_deg=2.0,
                           n_side=3, max_b=2000.0, seed=12, F=0, max_bin=6),
    "12ant": dict(n_ant=12, n_samp=1 << 14, dms=[4.0, 9.0, 20.0, 33.0], L=128, bw=8e6, field_deg=1.0,
                  n_side=5, max_b=4000.0, seed=13),
    "4ant_600blocks": dict(n_ant=4, n_samp=16 * 700 + 5, dms=[0.5, 2.0], L=16, bw=8e6, field_deg=1.0,
                           n_side=3, max_b=2000.0, seed=15),
    "24ant_276pairs": dict(n_ant=24, n_samp=4096, dms=[1.5, 6.0], L=64, bw=8e6, field_deg=1.0,
                           n_side=3, max_b=3000.0, seed=14, pulse=False),
}


def _oracle(cfg, x):
    return ocpi.search(x, cfg["xyz"], cfg["pix_lm"], cfg["f0"], cfg["bw"], K_DM, cfg["dms"],
                       cfg["blk_len"], cfg["half_width"], K=None if cfg["max_bin"] == 0 else cfg["max_bin"],
                       keep=True)


@pytest.mark.parametrize("mode", [0, 1], ids=["tensor_cores", "cuda_cores"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_spectra_and_image_match_the_oracle(name, mode):
    """image_mode 0: the dense split-BF16 image on the tensor cores (the
    default); 1: the sparse gathers on the CUDA cores.  Same tolerances."""
    cfg, x = _case(**CASES[name])
    E_o, kept, K_o = _oracle(cfg, x)
    with CpiPlan(cfg["xyz"], cfg["f0"], cfg["bw"], cfg["n_samp"], cfg["dms"], cfg["blk_len"],
                 cfg["pix_lm"], cfg["half_width"], cfg["max_bin"], k_dm=K_DM,
                 image_mode=mode) as plan:
        assert plan.max_bin == K_o
        nk = 2 * K_o + 1
        shape = (len(cfg["dms"]), plan.n_blk, nk, plan.n_pair)
        V = np.empty(shape, np.complex64)
        X = np.empty(shape, np.complex64)
        plan.spectra(x, V, X)
        E = np.empty((len(cfg["dms"]), plan.n_blk, plan.n_pix), np.float32)
        plan.run(x, E)
        kb = plan.layout(0)["pair_bins"]
        kb_o = ocpi.pair_bins(cfg["xyz"], cfg["pix_lm"], cfg["f0"], cfg["bw"], K_DM, cfg["dms"],
                              cfg["blk_len"], cfg["half_width"])
        assert np.array_equal(kb, kb_o)
        for d in range(len(cfg["dms"])):
            assert plan.layout(d)["n_win"] == ocpi.window_blocks(cfg["f0"], cfg["bw"], K_DM, cfg["dms"][d],
                                                                  cfg["blk_len"])
            Vo, Xo = kept[d]
            Vo = np.transpose(Vo, (1, 0, 2))  # oracle [bin][block][pair] -> [block][bin][pair]
            Xo = np.transpose(Xo, (1, 0, 2))
            ks = np.arange(-K_o, K_o + 1)
            need = np.abs(ks)[:, None] <= kb_o[None, :]          # [bin][pair]
            assert np.all(V[d][:, ~need] == 0) and np.all(X[d][:, ~need] == 0)
            ev = np.abs(V[d][:, need] - Vo[:, need]).max() / np.abs(Vo[:, need]).max()
            ex = np.abs(X[d][:, need] - Xo[:, need]).max() / max(np.abs(Xo[:, need]).max(), 1e-30)
            assert ev <= 2e-5, (d, ev)
            if np.abs(Xo).max() > 0:
                assert ex <= 2e-5, (d, ex)
            assert np.all(E[d][E_o[d] == 0] == 0)
            if E_o[d].max() > 0:
                ee = np.abs(E[d] - E_o[d]).max() / E_o[d].max()
                assert ee <= 1e-4, (d, ee)
        t = plan.timing()
        assert all(v >= 0 for v in t.values())


def test_device_and_host_buffers_agree_bit_for_bit():
    cfg, x = _case(**CASES["12ant"])
    with CpiPlan(cfg["xyz"], cfg["f0"], cfg["bw"], cfg["n_samp"], cfg["dms"], cfg["blk_len"],
                 cfg["pix_lm"], cfg["half_width"], k_dm=K_DM) as plan:
        Eh = np.empty((len(cfg["dms"]), plan.n_blk, plan.n_pix), np.float32)
        plan.run(x, Eh)
        Ed = torch.empty(Eh.shape, dtype=torch.float32, device="cuda")
        plan.run(torch.from_numpy(x).cuda(), Ed)
        assert np.array_equal(Eh, Ed.cpu().numpy())
        plan.run(x, Eh)  # repeatable
        assert np.array_equal(Eh, Ed.cpu().numpy())


def test_a_dispersed_burst_is_found_at_its_pixel_and_dm():
    """Sky-model burst (exact cold-plasma dispersion, noise-like emission) at a
    pixel centre: the brightest pixel of E is the burst's; per trial DM the
    peak over the median image level is highest at the trial DM nearest the
    truth (a longer window keeps the whole sweep but adds noise in proportion
    to its length, a shorter one cuts the sweep); at that DM the brightest
    window is centred near the sweep's temporal midpoint."""
    n_ant, n_samp, bw, f0, L = 12, 1 << 19, 32e6, 1.4e9, 2048
    xyz = skymodel.antenna_positions(n_ant, 6000.0, 21)
    pix = skymodel.pixel_grid(8, 1.0)
    dms = np.linspace(80.0, 120.0, 21)
    true_d, true_pix = 10, 43
    x = skymodel.noise(n_ant, n_samp, 22)
    p = skymodel.Pulse(dm=float(dms[true_d]), t0=0.55 * n_samp, fwhm_s=30e-6, amp=1.5,
                       l=pix[true_pix][0], m=pix[true_pix][1], seed=23)
    skymodel.inject(x, xyz, f0, bw, p)
    with CpiPlan(xyz, f0, bw, n_samp, dms, L, pix, 2, k_dm=K_DM) as plan:
        E = np.empty((len(dms), plan.n_blk, plan.n_pix), np.float32)
        plan.run(x, E)
        d, m, q = np.unravel_index(int(np.argmax(E)), E.shape)
        assert q == true_pix
        nws = [plan.layout(i)["n_win"] for i in range(len(dms))]
        ratio = [E[i, :, true_pix].max() / np.median(E[i, nws[i] - 1:, :]) for i in range(len(dms))]
        assert abs(int(np.argmax(ratio)) - true_d) <= 1
        assert max(ratio) > 100
        hi, lo = skymodel.sweep_samples(f0, bw, dms[true_d])
        mid = p.t0 + 0.5 * (lo - hi)                      # sweep's temporal midpoint, samples
        nw = nws[true_d]
        mt = int(np.argmax(E[true_d, :, true_pix]))
        centre = (mt + 1 - nw) * L + nw * L / 2
        assert abs(centre - mid) <= 2 * L


def test_sampled_windows_of_the_full_workload():
    """12 antennas within 6 km, 32 MHz at 1.4 GHz, 2^22 samples, 63 trial DMs in
    (0, 300], 32 x 32 beams over 1 degree, blocks of 2048: the GPU's X and E
    for a short and a long window of two DMs against the oracle computed on
    those windows' samples only."""
    sc = skymodel.chimageator_medium()
    dms = sc.dms[sc.dms > 0]
    x = sc.voltages()
    L, F = 2048, 2
    with CpiPlan(sc.xyz, sc.f0, sc.bw, sc.n_samp, dms, L, sc.pix_lm, F, k_dm=sc.k_dm) as plan:
        K = plan.max_bin
        nk = 2 * K + 1
        xd = torch.from_numpy(x).cuda()
        E = torch.empty((len(dms), plan.n_blk, plan.n_pix), dtype=torch.float32, device="cuda")
        plan.run(xd, E)
        Xd = torch.empty((len(dms), plan.n_blk, nk, plan.n_pair), dtype=torch.complex64, device="cuda")
        plan.spectra(xd, None, Xd)
        torch.cuda.synchronize()
        for d in (0, len(dms) - 1):
            nw = plan.layout(d)["n_win"]
            N = nw * L
            k0p, W = ocpi.image_weights(sc.xyz, sc.pix_lm, sc.f0, sc.bw, sc.k_dm, dms[d], L, F)
            for m in (nw - 1, (nw - 1 + plan.n_blk - 1) // 2):
                n0 = (m + 1 - nw) * L
                seg = ocpi.mix(x[:, n0:n0 + N])
                Xo = ocpi.cic(ocpi.partial_dft(seg, L, N, K), nw)[:, nw - 1, :]    # window's own time
                Eo = ocpi.image(Xo[:, None, :], k0p, W, K)[0]
                Xg = Xd[d, m].cpu().numpy()
                kb = plan.layout(d)["pair_bins"]
                need = np.abs(np.arange(-K, K + 1))[:, None] <= kb[None, :]
                assert np.abs(Xg[need] - Xo[need]).max() <= 2e-5 * np.abs(Xo[need]).max()
                Eg = E[d, m].cpu().numpy()
                assert np.abs(Eg - Eo).max() <= 1e-4 * Eo.max()
