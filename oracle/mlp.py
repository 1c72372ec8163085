"""FP64 statement of the surrogate network, its gradients and Adam.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The surrogate is not part of the paper; it seeds the bisection brackets of
the critical body force (Section 3.4).  Network: 5 inputs -> three hidden
layers of 128 SiLU units -> 2 outputs (mu, s), mu the predicted log g_crit
and s the log of the predicted variance.  Loss per sample (Gaussian negative
log-likelihood without the constant): 0.5 * (exp(-s) (y - mu)^2 + s),
averaged over the batch.  Parameters are stored flat in the order
W1 [128x5], b1 [128], W2 [128x128], b2, W3 [128x128], b3, W4 [2x128], b4 [2]
(row-major, out x in).  Adam as in Kingma & Ba (2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

SIZES = (5, 128, 128, 128, 2)


def n_params(sizes=SIZES) -> int:
    return sum(sizes[k + 1] * sizes[k] + sizes[k + 1] for k in range(len(sizes) - 1))


def unpack(theta, sizes=SIZES):
    out, o = [], 0
    for k in range(len(sizes) - 1):
        fan_in, fan_out = sizes[k], sizes[k + 1]
        W = theta[o:o + fan_out * fan_in].reshape(fan_out, fan_in)
        o += fan_out * fan_in
        b = theta[o:o + fan_out]
        o += fan_out
        out.append((W, b))
    return out


def init_params(seed: int, sizes=SIZES) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for k in range(len(sizes) - 1):
        fan_in, fan_out = sizes[k], sizes[k + 1]
        lim = 1.0 / np.sqrt(fan_in)
        parts.append(rng.uniform(-lim, lim, fan_out * fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(theta, x, sizes=SIZES):
    """x [B, 5] -> out [B, 2] (mu, s); also the layer inputs and pre-activations."""
    layers = unpack(np.asarray(theta, dtype=np.float64), sizes)
    a = np.asarray(x, dtype=np.float64)
    acts, zs = [a], []
    for k, (W, b) in enumerate(layers):
        z = a @ W.T + b
        zs.append(z)
        a = silu(z) if k < len(layers) - 1 else z
        acts.append(a)
    return a, acts, zs


def loss(theta, x, y, sizes=SIZES) -> float:
    out, _, _ = forward(theta, x, sizes)
    mu, s = out[:, 0], out[:, 1]
    r = np.asarray(y, dtype=np.float64) - mu
    return float(np.mean(0.5 * (np.exp(-s) * r * r + s)))


def grad(theta, x, y, sizes=SIZES):
    """(loss, dloss/dtheta) by the chain rule, layer by layer."""
    theta = np.asarray(theta, dtype=np.float64)
    layers = unpack(theta, sizes)
    out, acts, zs = forward(theta, x, sizes)
    B = out.shape[0]
    mu, s = out[:, 0], out[:, 1]
    r = np.asarray(y, dtype=np.float64) - mu
    e = np.exp(-s)
    L = float(np.mean(0.5 * (e * r * r + s)))
    d = np.empty_like(out)
    d[:, 0] = -e * r / B                     # dL/dmu
    d[:, 1] = 0.5 * (1.0 - e * r * r) / B    # dL/ds
    grads = [None] * len(layers)
    for k in range(len(layers) - 1, -1, -1):
        W, b = layers[k]
        if k < len(layers) - 1:
            d = d * dsilu(zs[k])
        gW = d.T @ acts[k]
        gb = d.sum(axis=0)
        grads[k] = (gW, gb)
        d = d @ W
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, flat


def adam_step(theta, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
