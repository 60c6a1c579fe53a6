"""The partial-sum recursion of the Chimageator's imaging step (App. B.2.1):
trials whose trajectories share a gradient (Eq. chimg_grad) *and* an
intercept lie on one line in dump-bin space, and each one's image is a
prefix of one cumulative sum along it.

Pins, all on the CPU against the FP64 oracle's own steps:
- the paper's model of Sec. 4.2 that the recursion assumes (a baseband chirp
  sweeping 0..B from the window start, Eq. chimg_xpq with its tau^2 term
  dropped) equals a simulated chirp put through mixing, gridding, the spatial
  DFT and integrate-and-dump, within the dropped term's bound, and its
  trajectory follows Eq. chimgf0 through k = 0 at the window start;
- on that model the recursion gives every trial of a line the image its own
  taps give (noise plus a perfect chirp, every window end);
- on the carrier-aware model the search uses (a chirp centred on its window,
  the carrier's spatial offset Ns tau a_0), two trials of equal gradient
  differ in intercept and taps, and reading the shorter from the longer's
  prefix loses most of a perfect chirp's energy: the search forms each
  trial's trajectory sum on its own."""
import math

import numpy as np

from oracle import chimg as oc
from oracle import cpi

B, L, NS, M, F = 8e6, 256, 16, 8, 1


def _paper_trial(n_win, rate):
    """(fdot, tau) of the trial of n_win dumps on the line `rate`."""
    T = n_win * L / B
    fdot = B / T
    return fdot, rate / fdot


def test_paper_model_equals_a_simulated_chirp_and_follows_chimgf0():
    rate = 0.25 * B / (NS * L)        # a quarter bin per dump
    n_win = 16
    fdot, tau = _paper_trial(n_win, rate)
    t = np.arange(n_win * L) / B
    y = np.exp(1j * math.pi * fdot * (t[None, :] - np.arange(M)[:, None] * tau) ** 2)
    Yp = oc.integrate(oc.spatial_dft(oc.mix_grid(y, "natural"), NS), L)
    # the dropped tau^2 phase, |pi fdot tau^2 (p^2 - (p+l)^2)| < pi fdot tau^2 M^2
    bound = math.pi * fdot * tau * tau * M * M
    assert bound < 0.05
    for r in range(n_win):
        yh = oc.paper_expected_y(M, rate, B, L, NS, r)
        assert np.abs(Yp[:, r] - yh).max() <= bound * (M - 1) * L
        # Eq. chimgf0: k_0 = Ns fdot tau n / f_s, through k = 0 at the start
        k0 = NS * rate * (r * L + (L - 1) / 2.0) / B
        assert int(np.argmax(np.abs(yh))) == int(np.rint(k0)) % NS
    assert int(np.argmax(np.abs(oc.paper_expected_y(M, rate, B, L, NS, 0)))) == 0


def test_recursion_reproduces_each_trials_own_image_on_the_paper_model():
    rate = 0.3 * B / (NS * L)
    n_wins = [3, 5, 8, 13]
    rng = np.random.default_rng(5)
    n_dump = 24
    y = (rng.standard_normal((M, n_dump * L)) + 1j * rng.standard_normal((M, n_dump * L))) * 0.3
    # a perfect chirp of the 8-dump trial starting at dump 6
    fdot, tau = _paper_trial(8, rate)
    t = np.arange(8 * L) / B
    y[:, 6 * L:14 * L] += np.exp(1j * math.pi * fdot * (t[None, :] - np.arange(M)[:, None] * tau) ** 2)
    Y = oc.integrate(oc.spatial_dft(oc.mix_grid(y, "natural"), NS), L)
    Ed = oc.paper_image_direct(Y, M, rate, n_wins, B, L, NS, F)
    Es = oc.paper_image_shared(Y, M, rate, n_wins, B, L, NS, F)
    assert np.abs(Es - Ed).max() <= 1e-12 * Ed.max()
    # the chirp's own trial peaks where its window ends
    assert int(np.argmax(Ed[2])) == 13


def test_equal_gradient_trials_of_the_carrier_aware_model_do_not_share_prefixes():
    f0, D, kdm = 1.4e9, 500.0, 4.148808e15
    dm1, dm2 = 20.0, 40.0
    n1 = cpi.window_blocks(f0, B, kdm, dm1, L)
    n2 = cpi.window_blocks(f0, B, kdm, dm2, L)
    assert n2 > n1 > 4
    _, _, a1_1 = cpi.chirp_model(f0, B, kdm, dm1)
    _, _, a1_2 = cpi.chirp_model(f0, B, kdm, dm2)
    l1 = 0.012                                   # ~0.17 bins per dump
    l2 = l1 * a1_1 / a1_2                        # equal gradient tau a_1 (Eq. chimg_grad)
    g1 = NS * D * l1 / oc.C_LIGHT * a1_1 * L / B
    g2 = NS * D * l2 / oc.C_LIGHT * a1_2 * L / B
    assert abs(g1 - g2) <= 1e-12 * abs(g1) and 0.1 < abs(g1) < 0.5

    def taps(dm, ld, n):
        out = []
        for r in range(n):
            yh = oc.expected_y(M, D, ld, f0, B, kdm, dm, L, NS, r)
            kc = oc.trajectory_bins(D, ld, f0, B, kdm, dm, L, NS, r)
            ks = [(kc + j) % NS for j in range(-F, F + 1)]
            out.append((ks, np.conj(yh[ks]) / ((M - 1) * L)))
        return out

    t1, t2 = taps(dm1, l1, n1), taps(dm2, l2, n2)
    # the intercepts differ: the bin sequences of the shared dumps disagree
    assert any(t1[r][0] != t2[r][0] for r in range(n1))
    # a perfect chirp of trial 1: its own taps against the longer trial's prefix
    Y = np.stack([oc.expected_y(M, D, l1, f0, B, kdm, dm1, L, NS, r) for r in range(n1)], axis=1)
    own = abs(oc.prefix_sums(Y, t1, 0)[-1]) ** 2
    shared = abs(oc.prefix_sums(Y, t2[:n1], 0)[-1]) ** 2
    assert shared < 0.5 * own, (shared, own)
