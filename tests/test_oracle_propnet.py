"""Pins of the proposal-network oracle: the convolution against scipy's
cross-correlation (an independent library), every parameter gradient against
FP64 central differences, the BCE gradient against its closed form, and the
first Adam step against its closed form (a sign step of size lr)."""
import numpy as np
import pytest

from oracle import propnet as pn

signal = pytest.importorskip("scipy.signal")


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    B, C, O, T, K = 2, 3, 4, 17, 5
    x = rng.standard_normal((B, C, T))
    W = rng.standard_normal((O, C, K))
    b = rng.standard_normal(O)
    out = pn.conv(x, W, b, K // 2)
    for bb in range(B):
        for o in range(O):
            ref = b[o] + sum(signal.correlate(x[bb, i], W[o, i], mode="same") for i in range(C))
            assert np.allclose(out[bb, o], ref, atol=1e-12)


@pytest.mark.parametrize("n_dm,hidden,k1,k2", [(3, 4, 3, 3), (5, 3, 5, 1)])
def test_gradients_match_central_differences(n_dm, hidden, k1, k2):
    rng = np.random.default_rng(2)
    B, T = 2, 11
    theta = pn.init(n_dm, hidden, k1, k2, 3) + 0.05 * rng.standard_normal(
        pn.n_params(n_dm, hidden, k1, k2))
    x = rng.standard_normal((B, n_dm, T))
    y = (rng.random((B, n_dm, T)) < 0.2).astype(float)
    loss, g = pn.loss_and_grad(theta, x, y, 4.0, n_dm, hidden, k1, k2)
    h = 1e-6
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = pn.loss_and_grad(tp, x, y, 4.0, n_dm, hidden, k1, k2)
        lm, _ = pn.loss_and_grad(tm, x, y, 4.0, n_dm, hidden, k1, k2)
        assert abs((lp - lm) / (2 * h) - g[i]) < 1e-7 + 1e-5 * abs(g[i]), i


def test_bce_closed_form():
    z = np.array([-3.0, 0.0, 2.5])
    y = np.array([1.0, 0.0, 1.0])
    loss, dz = pn.bce(z, y, 2.0)
    s = 1 / (1 + np.exp(-z))
    expect = (2.0 * np.log1p(np.exp(3.0)) + np.log(2.0) + 2.0 * np.log1p(np.exp(-2.5))) / 3
    assert loss == pytest.approx(expect, rel=1e-14)
    assert np.allclose(dz, np.array([2.0 * (s[0] - 1), s[1], 2.0 * (s[2] - 1)]) / 3, rtol=1e-14)


def test_first_adam_step_is_a_sign_step():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 2.0])
    t1, m, v = pn.adam(theta, g, np.zeros(3), np.zeros(3), 1, 0.01, eps=0.0)
    assert np.allclose(t1, theta - 0.01 * np.sign(g), rtol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
