"""CPU check of the method the CUDA pre-integrator uses to evaluate the
partial DFTs (Sec. A.3.2), restated in FP64 numpy: per sub-block of Ls
samples, J moments t_j = (-j)^j / j! sum_i u_i^j x_i, u = (i - c)/(Ls/2),
and V(f) = sum_s exp(-2 pi j c_s f) sum_j theta^j t_j, theta = pi f Ls, with
Ls the largest power of two <= min(L, 256) giving theta <= 1/2 at the highest
frequency and J the smallest with theta^J / J! <= 1e-9.  Against the
oracle's direct sums the truncation must stay below 1e-8 of the block scale
for every regime the plan can pick (tiny blocks, many bins, long windows)."""
import math

import numpy as np
import pytest

from oracle import cpi


def _plan_terms(L, fmax):
    Ls = min(L, 256)
    while Ls > 1 and math.pi * fmax * Ls > 0.5:
        Ls //= 2
    th = math.pi * fmax * Ls
    J, t = 1, th
    if Ls > 1 and th > 0:
        while t > 1e-9 and J < 12:
            J += 1
            t *= th / J
    return Ls, J


def _taylor_partial(x, L, Ls, J, k, n_win):
    g = math.gcd(k, n_win)
    kp, npr = k // g, n_win // g
    f = kp / (npr * L)
    th = math.pi * f * Ls
    n_blk = x.shape[1] // L
    u = (2 * np.arange(Ls) - Ls + 1) / Ls
    V = np.zeros((n_blk, x.shape[0]), complex)
    for m in range(n_blk):
        for sl in range(L // Ls):
            s = m * (L // Ls) + sl
            seg = x[:, s * Ls:(s + 1) * Ls]
            poly = sum(((-1j) ** j) / math.factorial(j) * (seg * u ** j).sum(1) * th ** j for j in range(J))
            c = s * Ls + (Ls - 1) / 2
            V[m] += np.exp(-2j * math.pi * c * f) * poly
    return V


@pytest.mark.parametrize("L,K,n_win", [(16, 2, 1), (64, 8, 1), (256, 6, 3), (2048, 8, 7), (128, 40, 2)])
def test_taylor_partial_dfts_match_direct_sums(L, K, n_win):
    rng = np.random.default_rng(L + K)
    x = rng.standard_normal((3, 6 * L)) + 1j * rng.standard_normal((3, 6 * L))
    Ls, J = _plan_terms(L, K / (n_win * L))
    assert math.pi * K / (n_win * L) * Ls <= 0.5 or Ls == 1
    Vo = cpi.partial_dft(x, L, n_win * L, K)
    scale = np.abs(Vo).max()
    for k in (1, K // 2 + 1, K):
        got = _taylor_partial(x, L, Ls, J, k, n_win)
        assert np.abs(got - Vo[K + k]).max() <= 1e-8 * scale, (k, Ls, J)
