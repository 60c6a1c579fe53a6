"""FP64 numpy oracle of the proposal network (test infrastructure only).

The network reads the incoherent dedispersed power of the antenna-incoherent
search (Sec. 2.3.1), normalised per trial DM, as a 1-D signal over time with
the DM grid as channels, and returns one logit per (trial DM, time sample):

  h1 = relu(conv(x,  W1, b1, pad = K1 // 2))      [B, H, T]
  h2 = relu(conv(h1, W2, b2, pad = K2 // 2))      [B, H, T]
  z  =      conv(h2, W3, b3, pad = 0),  K3 = 1    [B, C, T]

with conv(x, W, b, pad)[b, o, t] = b[o] + sum_{i,k} W[o, i, k] x[b, i, t + k - pad]
(zero outside [0, T)).  Loss: mean over all elements of the class-weighted
binary cross-entropy with logits,
  l = p y softplus(-z) + (1 - y) softplus(z),  p = positive-class weight,
and Adam (Kingma & Ba, 2015) updates.  Parameters travel as one flat vector in
the order W1, b1, W2, b2, W3, b3.

Written for checking by eye: explicit sums, no fusion.
"""

from __future__ import annotations

import numpy as np


def shapes(n_dm: int, hidden: int, k1: int, k2: int):
    return [(hidden, n_dm, k1), (hidden,), (hidden, hidden, k2), (hidden,), (n_dm, hidden, 1),
            (n_dm,)]


def n_params(n_dm, hidden, k1, k2) -> int:
    return int(sum(np.prod(s) for s in shapes(n_dm, hidden, k1, k2)))


def unflatten(theta, n_dm, hidden, k1, k2):
    out, o = [], 0
    for s in shapes(n_dm, hidden, k1, k2):
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def flatten(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def conv(x, W, b, pad):
    """conv(x, W, b, pad)[b, o, t] = b[o] + sum_{i,k} W[o,i,k] x[b, i, t + k - pad]."""
    B, C, T = x.shape
    O, _, K = W.shape
    xp = np.zeros((B, C, T + K - 1))
    xp[:, :, pad:pad + T] = x
    out = np.zeros((B, O, T)) + b[None, :, None]
    for k in range(K):
        out += np.einsum("oi,bit->bot", W[:, :, k], xp[:, :, k:k + T])
    return out


def forward(theta, x, n_dm, hidden, k1, k2):
    W1, b1, W2, b2, W3, b3 = unflatten(theta, n_dm, hidden, k1, k2)
    a1 = conv(x, W1, b1, k1 // 2)
    h1 = np.maximum(a1, 0.0)
    a2 = conv(h1, W2, b2, k2 // 2)
    h2 = np.maximum(a2, 0.0)
    z = conv(h2, W3, b3, 0)
    return z, (x, a1, h1, a2, h2)


def softplus(z):
    return np.logaddexp(0.0, z)


def bce(z, y, pos_weight):
    """Mean class-weighted BCE with logits and its gradient d loss / d z."""
    n = z.size
    loss = (pos_weight * y * softplus(-z) + (1.0 - y) * softplus(z)).sum() / n
    s = 1.0 / (1.0 + np.exp(-z))
    dz = (-pos_weight * y * (1.0 - s) + (1.0 - y) * s) / n
    return loss, dz


def conv_backward(x, W, pad, g):
    """Gradients of conv with respect to x, W and b given g = d loss / d out."""
    B, C, T = x.shape
    O, _, K = W.shape
    xp = np.zeros((B, C, T + K - 1))
    xp[:, :, pad:pad + T] = x
    dW = np.zeros_like(W)
    dxp = np.zeros_like(xp)
    for k in range(K):
        dW[:, :, k] = np.einsum("bot,bit->oi", g, xp[:, :, k:k + T])
        dxp[:, :, k:k + T] += np.einsum("oi,bot->bit", W[:, :, k], g)
    db = g.sum(axis=(0, 2))
    return dxp[:, :, pad:pad + T], dW, db


def loss_and_grad(theta, x, y, pos_weight, n_dm, hidden, k1, k2):
    W1, b1, W2, b2, W3, b3 = unflatten(theta, n_dm, hidden, k1, k2)
    z, (x0, a1, h1, a2, h2) = forward(theta, x, n_dm, hidden, k1, k2)
    loss, dz = bce(z, y, pos_weight)
    dh2, dW3, db3 = conv_backward(h2, W3, 0, dz)
    da2 = dh2 * (a2 > 0)
    dh1, dW2, db2 = conv_backward(h1, W2, k2 // 2, da2)
    da1 = dh1 * (a1 > 0)
    _, dW1, db1 = conv_backward(x0, W1, k1 // 2, da1)
    return loss, flatten([dW1, db1, dW2, db2, dW3, db3])


def adam(theta, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns new theta, m, v."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init(n_dm, hidden, k1, k2, seed):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes(n_dm, hidden, k1, k2):
        if len(s) == 3:
            fan_in = s[1] * s[2]
            parts.append(rng.standard_normal(s) * np.sqrt(2.0 / fan_in))
        else:
            parts.append(np.zeros(s))
    return flatten(parts)
