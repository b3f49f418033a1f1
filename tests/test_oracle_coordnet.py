"""Pins for the FP64 oracle of the surrogate's coordinate network
(oracle/coordnet.py): row inputs at cases with closed forms (normal incidence,
past the critical angle, the mirror symmetry of the tilt), exact feature
values, forward against an independent torch.nn.functional restatement,
backward against central differences, and the image assembly against the
demodulation it inverts."""
import math

import numpy as np
import pytest

from oracle import coordnet as cn

WIN = {"x0": -20e-3, "x1": 20e-3, "z0": 0.0, "z1": 40e-3, "nx": 128, "nz": 128}
LO = (0.0, 20e-3, 2e6, 1e-3)
HI = (math.radians(15.0), 60e-3, 10e6, 20e-3)
C1, C2, A = 1480.0, 5900.0, 6.35e-3


def test_row_inputs_at_normal_incidence():
    # tilt 0: the refracted axis is the z axis (th = 0), s = z, t = x
    p = [[3e-3, 0.0, 40e-3, 5e6, 10e-3]]
    i, j = 100, 17
    c = cn.row_inputs(p, [i], [j], WIN, LO, HI, C1, C2, A)[0]
    x = -20e-3 + (i + 0.5) * 40e-3 / 128
    zw = (j + 0.5) * 40e-3 / 128
    z = 10e-3 + zw
    q = A * A * 5e6 / (C1 * (40e-3 + (C2 / C1) * z))
    want = [-1.0, 0.0, -0.25, 2 * (10e-3 - 1e-3) / 19e-3 - 1.0, x / 20e-3, 2 * zw / 40e-3 - 1.0,
            z / 20e-3, x / 20e-3, math.log(q)]
    assert np.allclose(c, want, rtol=0, atol=1e-14)


def test_row_inputs_past_the_critical_angle_and_mirror():
    crit = math.asin(C1 / C2)
    p = [[0.0, crit + 0.01, 30e-3, 3e6, 5e-3]]
    i, j = 3, 90
    c = cn.row_inputs(p, [i], [j], WIN, LO, HI, C1, C2, A)[0]
    x = -20e-3 + (i + 0.5) * 40e-3 / 128
    z = 5e-3 + (j + 0.5) * 40e-3 / 128
    # th = pi/2: s = x, t = -z; the Fresnel path clamps s < 0 to 0
    assert c[6] == pytest.approx(x / 20e-3, abs=1e-15)
    assert c[7] == pytest.approx(-z / 20e-3, abs=1e-15)
    assert c[8] == pytest.approx(math.log(A * A * 3e6 / (C1 * 30e-3)), abs=1e-14)
    # mirror: tilt -> -tilt with pixel i -> nx - 1 - i gives the same inputs
    rng = np.random.default_rng(0)
    for _ in range(20):
        tilt = rng.uniform(0, 0.26)
        pp = [[rng.uniform(-1e-2, 1e-2), tilt, rng.uniform(0.02, 0.06), rng.uniform(2e6, 1e7), 0.01]]
        pm = [[pp[0][0], -tilt] + pp[0][2:]]
        i, j = rng.integers(0, 128), rng.integers(0, 128)
        a = cn.row_inputs(pp, [i], [j], WIN, LO, HI, C1, C2, A)
        b = cn.row_inputs(pm, [127 - i], [j], WIN, LO, HI, C1, C2, A)
        assert np.allclose(a, b, rtol=0, atol=1e-15)  # x0 + (i + 1/2) dx mirrors to rounding


def test_features_at_hand_picked_inputs():
    c = np.zeros((2, 9))
    c[0, 0], c[0, 1] = 1.0, 0.5
    c[1, 8] = -1.0
    B = np.zeros((3, 9))
    B[0, 0] = 1.0           # pi c0
    B[1, 1] = 1.0           # pi c1
    B[2, 0], B[2, 8] = 0.5, 2.0
    f = cn.features(c, B)
    assert f.shape == (2, 6 + 16)
    args = np.pi * np.array([[1.0, 0.5, 0.5], [0.0, 0.0, -2.0]])
    exact = np.array([[0, 1, 1, -1, 0, 0], [0, 0, 0, 1, 1, 1]], dtype=np.float64)
    assert np.allclose(np.concatenate([np.sin(args), np.cos(args)], 1), exact, atol=1e-15)
    assert np.allclose(f[:, :6], exact, atol=1e-15)
    assert np.array_equal(f[:, 6:15], c) and np.all(f[:, 15:] == 0)


def tiny_net(rng, K0=22, width=7, depth=2):
    sizes = [K0] + [width] * depth + [3]
    W = [rng.normal(size=(sizes[i + 1], sizes[i])) / np.sqrt(sizes[i]) for i in range(len(sizes) - 1)]
    b = [rng.normal(size=sizes[i + 1]) * 0.1 for i in range(len(sizes) - 1)]
    return {"W": W, "b": b}


def test_forward_matches_an_independent_torch_restatement():
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(1)
    params = tiny_net(rng, depth=3)
    B = rng.normal(size=(3, 9))
    h0 = cn.features(rng.normal(size=(5, 9)), B)
    y, _ = cn.forward(params, h0)
    t = lambda a: torch.tensor(a, dtype=torch.float64)
    h = t(h0)
    for W, b in zip(params["W"][:-1], params["b"][:-1]):
        h = F.silu(F.linear(h, t(W), t(b)))
    want = F.linear(h, t(params["W"][-1]), t(params["b"][-1])).numpy()
    assert y.shape == (5, 3)
    assert np.allclose(y, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_backward_matches_central_differences():
    rng = np.random.default_rng(2)
    params = tiny_net(rng)
    h0 = rng.normal(size=(6, 22))
    tgt = rng.normal(size=(6, 3))
    y, cache = cn.forward(params, h0)
    g = cn.backward(params, cache, y, tgt)
    eps = 1e-6
    for kind in ("W", "b"):
        for l, arr in enumerate(params[kind]):
            flat = arr.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[idx]
                flat[idx] = old + eps
                lp = cn.loss(cn.forward(params, h0)[0], tgt)
                flat[idx] = old - eps
                lm = cn.loss(cn.forward(params, h0)[0], tgt)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - g[kind][l].reshape(-1)[idx]) <= 1e-7 * max(1.0, abs(fd)), (kind, l, idx)


def test_image_inverts_the_demodulation():
    # rows (re, im, log rms) built from a synthetic image by the targets'
    # definition (times exp(-i psi), over the RMS) give back that image
    win = dict(WIN, nx=16, nz=12)
    p = (2e-3, math.radians(-7.0), 35e-3, 4e6, 6e-3)
    rng = np.random.default_rng(3)
    img = rng.normal(size=(12, 16)) + 1j * rng.normal(size=(12, 16))
    _, tilt, L, f, d = p
    k1, k2 = 2 * math.pi * f / C1, 2 * math.pi * f / C2
    S = (C2 / C1) * math.sin(tilt)
    Cc = math.sqrt(1 - S * S)
    x = -20e-3 + (np.arange(16) + 0.5) * 40e-3 / 16
    z = d + (np.arange(12) + 0.5) * 40e-3 / 12
    psi = k1 * L + k2 * (S * x[None, :] + Cc * z[:, None])
    env = img * np.exp(-1j * psi)
    rms = math.sqrt(np.mean(np.abs(env) ** 2))
    rows = np.stack([(env / rms).real.ravel(), (env / rms).imag.ravel(), np.full(env.size, math.log(rms))], 1)
    assert np.allclose(cn.image(rows, p, win, C1, C2), img, rtol=0, atol=1e-12)
    # a unit envelope is the plane wave itself: |image| = 1, phase psi
    ones = np.stack([np.ones(192), np.zeros(192), np.zeros(192)], 1)
    pw = cn.image(ones, p, win, C1, C2)
    assert np.allclose(np.abs(pw), 1.0) and np.allclose(pw, np.exp(1j * psi))
