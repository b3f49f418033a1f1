"""FP64 CPU oracle of the learned surrogate's coordinate network.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy in float64;
shares no code with the CUDA path.  The surrogate is not in the paper: it
maps the inputs of one water -> steel chain (transducer x-offset, tilt, water
path L along the axis, frequency f, image depth d) to the field image the
RSI chain computes (Sec. 2.1).  Its network is evaluated per PIXEL: one row
per (field, pixel) with inputs built from the field's parameters and the
pixel's position, and three outputs -- the real and imaginary part of the
pixel's envelope (the image times exp(-i psi), psi the refracted plane wave's
phase) divided by the field's RMS envelope, and the log of that RMS.

Row inputs c (9 values) of field p = (x_off, tilt, L, f, d), pixel (i, j) of
the window {x0, x1, z0, z1, nx, nz} (x relative to the point where the axis
meets the interface, z below the window's top edge, which lies d below the
interface; Wx = x1 - x0, Wz = z1 - z0):
    sg = sign(tilt) (+1 at 0), a1 = |tilt|          (mirror symmetry x -> -x)
    xw = x0 + (i + 1/2) Wx / nx,  zw = z0 + (j + 1/2) Wz / nz
    x  = sg xw,  z = d + zw
    th = asin(min(1, (c2 / c1) sin a1))              (Snell's law, Eq. root_searching)
    s  = x sin th + z cos th,  t = x cos th - z sin th   (along / across the refracted axis)
    q  = a^2 f / (c1 (L + (c2 / c1) max(s, 0)))      (Fresnel number of the equivalent path)
    c  = [n(a1), n(L), n(f), n(d), x / S0, 2 (zw - z0) / Wz - 1, s / S0, t / S0, ln q]
with n(v) = 2 (v - lo) / (hi - lo) - 1 over the box of (|tilt|, L, f, d) and
S0 = Wx / 2.
The x-offset does not enter: shifting the transducer shifts the interface patch
and the window with it, so the field in window coordinates does not change.

Network:
    h0 = [sin(pi B c), cos(pi B c), c, 0 ...]      (B: F x 9; 2F + 16 values)
    h_l = silu(W_l h_{l-1} + b_l), l = 1..depth
    y = W_out h_depth + b_out                       (3 outputs)
    loss = sum over rows and the 3 outputs of (y - t)^2 / (4 rows)
(the divisor 4 counts the 4 slots of a row, the fourth always 0 on both sides).

backward() is the chain rule for that definition.  Pins: tests/test_oracle_coordnet.py.
"""
from __future__ import annotations

import math

import numpy as np

N_IN = 9
RAW = 16  # raw inputs appended to the Fourier features, zero-padded to 16


def row_inputs(p, i, j, window: dict, box_lo, box_hi, c1: float, c2: float, a: float):
    """The 9 row inputs c for fields p [rows, 5] at pixels (i, j) [rows]."""
    p = np.atleast_2d(np.asarray(p, np.float64))
    i = np.asarray(i, np.float64)
    j = np.asarray(j, np.float64)
    x0, x1, z0, z1 = (float(window[k]) for k in ("x0", "x1", "z0", "z1"))
    nx, nz = int(window["nx"]), int(window["nz"])
    Wx, Wz = x1 - x0, z1 - z0
    tilt, L, f, d = p[:, 1], p[:, 2], p[:, 3], p[:, 4]
    sg = np.where(tilt < 0.0, -1.0, 1.0)
    a1 = np.abs(tilt)
    xw = x0 + (i + 0.5) * Wx / nx
    zw = z0 + (j + 0.5) * Wz / nz
    x = sg * xw
    z = d + zw
    th = np.arcsin(np.minimum(1.0, (c2 / c1) * np.sin(a1)))
    s = x * np.sin(th) + z * np.cos(th)
    t = x * np.cos(th) - z * np.sin(th)
    q = a * a * f / (c1 * (L + (c2 / c1) * np.maximum(s, 0.0)))
    lo, hi = np.asarray(box_lo, np.float64), np.asarray(box_hi, np.float64)
    n = lambda v, k: 2.0 * (v - lo[k]) / (hi[k] - lo[k]) - 1.0
    S0 = 0.5 * Wx
    return np.stack([n(a1, 0), n(L, 1), n(f, 2), n(d, 3), x / S0, 2.0 * (zw - z0) / Wz - 1.0,
                     s / S0, t / S0, np.log(q)], axis=1)


def features(c, B):
    """[rows, 9] inputs -> [rows, 2F + 16] network inputs."""
    c = np.asarray(c, np.float64)
    arg = np.pi * (c @ np.asarray(B, np.float64).T)
    pad = np.zeros((c.shape[0], RAW - N_IN))
    return np.concatenate([np.sin(arg), np.cos(arg), c, pad], axis=1)


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params: dict, h0):
    """params: {"W": [W_1..W_depth, W_out], "b": [...]} (W: out x in);
    returns y [rows, 3] and the cache for backward()."""
    h = np.asarray(h0, np.float64)
    hs, zs = [h], []
    for W, b in zip(params["W"][:-1], params["b"][:-1]):
        z = h @ W.T + b
        zs.append(z)
        h = silu(z)
        hs.append(h)
    y = h @ params["W"][-1].T + params["b"][-1]
    return y, (hs, zs)


def loss(y, t):
    return float(np.sum((np.asarray(y) - np.asarray(t)) ** 2) / (4.0 * y.shape[0]))


def backward(params: dict, cache, y, t):
    """Gradients of loss() with respect to every W and b."""
    hs, zs = cache
    Ws = params["W"]
    dy = 2.0 * (np.asarray(y) - np.asarray(t)) / (4.0 * y.shape[0])
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


def image(y_rows, p, window: dict, c1: float, c2: float):
    """The field image [nz, nx] from the rows of one field (row = j nx + i):
    exp(mean of the log-RMS outputs) (re + i im) exp(i psi), psi = k1 L +
    k2 (S x + C z) the refracted plane wave's phase (S = (c2/c1) sin(tilt),
    C = sqrt(max(0, 1 - S^2)); x from the axis hit point, z = d + zw below the
    interface)."""
    y_rows = np.asarray(y_rows, np.float64)
    x0, x1, z0, z1 = (float(window[k]) for k in ("x0", "x1", "z0", "z1"))
    nx, nz = int(window["nx"]), int(window["nz"])
    _, tilt, L, f, d = (float(v) for v in p)
    k1, k2 = 2 * math.pi * f / c1, 2 * math.pi * f / c2
    S = (c2 / c1) * math.sin(tilt)
    C = math.sqrt(max(0.0, 1.0 - S * S))
    x = x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx
    z = d + z0 + (np.arange(nz) + 0.5) * (z1 - z0) / nz
    psi = k1 * L + k2 * (S * x[None, :] + C * z[:, None])
    env = (y_rows[:, 0] + 1j * y_rows[:, 1]).reshape(nz, nx)
    return math.exp(float(np.mean(y_rows[:, 2]))) * env * np.exp(1j * psi)
