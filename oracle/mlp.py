"""FP64 CPU oracle of the learned surrogate (a Fourier-feature MLP).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy in float64;
shares no code with the CUDA path.  The surrogate is not in the paper: it
maps transducer offset, tilt, water path, frequency and image depth to the
field image the RSI chain computes (Sec. 2.1), and is defined here as:

    u      = 2 (p - lo) / (hi - lo) - 1                     (inputs to [-1, 1])
    h0     = [sin(pi B u), cos(pi B u)]                     (Fourier features, B: F x n_in)
    z_l    = W_l h_{l-1} + b_l,  h_l = silu(z_l), l = 1..L  (silu(z) = z / (1 + e^-z))
    y      = W_out h_L + b_out
    loss   = mean over batch and outputs of (y - t)^2

backward() is the chain rule written out for that definition; adam_step()
follows Kingma & Ba (2015), Algorithm 1.  Pins: tests/test_oracle_mlp.py
(central finite differences, torch.optim.Adam).
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def features(p, lo, hi, B):
    """[batch, n_in] parameters -> [batch, 2F] Fourier features."""
    u = 2.0 * (np.asarray(p, np.float64) - lo) / (hi - lo) - 1.0
    a = np.pi * (u @ np.asarray(B, np.float64).T)
    return np.concatenate([np.sin(a), np.cos(a)], axis=1)


def forward(params: dict, p, lo, hi, B):
    """params: {"W": [W_1..W_L, W_out], "b": [...]} (W_l: out x in).
    Returns y and the cache for backward()."""
    h = features(p, lo, hi, B)
    hs, zs = [h], []
    Ws, bs = params["W"], params["b"]
    for l in range(len(Ws) - 1):
        z = h @ Ws[l].T + bs[l]
        zs.append(z)
        h = silu(z)
        hs.append(h)
    y = h @ Ws[-1].T + bs[-1]
    return y, (hs, zs)


def loss(y, t):
    return float(np.mean((y - t) ** 2))


def backward(params: dict, cache, y, t):
    """Gradients of loss() with respect to every W and b."""
    hs, zs = cache
    Ws = params["W"]
    n = y.size
    dy = 2.0 * (y - t) / n
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    gW[-1] = dy.T @ hs[-1]
    gb[-1] = dy.sum(axis=0)
    dh = dy @ Ws[-1]
    for l in range(len(Ws) - 2, -1, -1):
        dz = dh * silu_grad(zs[l])
        gW[l] = dz.T @ hs[l]
        gb[l] = dz.sum(axis=0)
        dh = dz @ Ws[l]
    return {"W": gW, "b": gb}


def adam_step(w, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1); returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v
