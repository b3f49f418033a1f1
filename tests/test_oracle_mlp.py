"""Pins for the FP64 surrogate oracle (oracle/mlp.py): backward() against
central finite differences of loss() on a tiny network, Adam against
torch.optim.Adam (FP64, CPU), and the silu derivative against differences."""
import numpy as np
import pytest

from oracle import mlp


def tiny_net(rng, n_in=5, F=3, width=7, depth=2, n_out=4):
    sizes = [2 * F] + [width] * depth + [n_out]
    W = [rng.normal(size=(sizes[i + 1], sizes[i])) / np.sqrt(sizes[i]) for i in range(len(sizes) - 1)]
    b = [rng.normal(size=sizes[i + 1]) * 0.1 for i in range(len(sizes) - 1)]
    B = rng.normal(size=(F, n_in))
    return {"W": W, "b": b}, B


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, rtol=1e-8, atol=1e-10)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    params, B = tiny_net(rng)
    lo, hi = -np.ones(5), 2 * np.ones(5)
    p = rng.uniform(-1, 2, size=(6, 5))
    t = rng.normal(size=(6, 4))
    y, cache = mlp.forward(params, p, lo, hi, B)
    g = mlp.backward(params, cache, y, t)
    h = 1e-6
    for kind in ("W", "b"):
        for l, arr in enumerate(params[kind]):
            flat = arr.reshape(-1)
            for idx in range(0, flat.size, max(1, flat.size // 7)):
                old = flat[idx]
                flat[idx] = old + h
                lp = mlp.loss(mlp.forward(params, p, lo, hi, B)[0], t)
                flat[idx] = old - h
                lm = mlp.loss(mlp.forward(params, p, lo, hi, B)[0], t)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = g[kind][l].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-7 * max(1.0, abs(fd)), (kind, l, idx, fd, an)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    w0 = rng.normal(size=50)
    grads = [rng.normal(size=50) for _ in range(5)]
    t = torch.tensor(w0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for step, g in enumerate(grads, start=1):
        opt.zero_grad()
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        w, m, v = mlp.adam_step(w, g, m, v, step, 3e-3)
    assert np.allclose(w, t.detach().numpy(), rtol=0, atol=1e-14)


def test_features_range_and_periodicity():
    rng = np.random.default_rng(2)
    B = rng.normal(size=(4, 5))
    lo, hi = np.zeros(5), np.ones(5)
    p = rng.uniform(size=(3, 5))
    f = mlp.features(p, lo, hi, B)
    assert f.shape == (3, 8)
    assert np.allclose(f[:, :4] ** 2 + f[:, 4:] ** 2, 1.0)


def test_forward_matches_an_independent_torch_restatement():
    """forward() against the network built from torch.nn.functional in FP64
    (linear layers, F.silu, sin/cos features) with the same weights: a
    dropped pi, a wrong input normalisation, a missing bias or SiLU on the
    output layer would all show here."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    rng = np.random.default_rng(3)
    params, B = tiny_net(rng, F=4, width=9, depth=3, n_out=6)
    lo = np.array([-2.0, 0.0, 1.0, -1.0, 5.0])
    hi = np.array([3.0, 0.5, 4.0, 1.0, 9.0])
    p = lo + (hi - lo) * rng.uniform(size=(7, 5))
    y, _ = mlp.forward(params, p, lo, hi, B)

    t = lambda a: torch.tensor(a, dtype=torch.float64)
    x = (t(p) - t(lo)) / (t(hi) - t(lo)) * 2.0 - 1.0
    arg = torch.pi * F.linear(x, t(B))
    h = torch.cat([torch.sin(arg), torch.cos(arg)], dim=1)
    for W, b in zip(params["W"][:-1], params["b"][:-1]):
        h = F.silu(F.linear(h, t(W), t(b)))
    want = F.linear(h, t(params["W"][-1]), t(params["b"][-1])).numpy()
    assert np.allclose(y, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_features_at_hand_picked_inputs():
    """Exact feature values: inputs at lo, hi and the middle of the box map
    to u = -1, 1, 0; with integer and half-integer rows of B the arguments
    pi B u are multiples of pi/2, whose sines and cosines are 0 and +-1."""
    lo = np.array([0.0, -1.0])
    hi = np.array([2.0, 3.0])
    B = np.array([[1.0, 0.0],    # pi u1
                  [0.0, 0.5],    # pi u2 / 2
                  [1.0, 1.0]])   # pi (u1 + u2)
    p = np.array([[0.0, -1.0],   # u = (-1, -1)
                  [2.0, 3.0],    # u = ( 1,  1)
                  [1.0, 1.0],    # u = ( 0,  0)
                  [0.0, 3.0]])   # u = (-1,  1)
    f = mlp.features(p, lo, hi, B)
    want_arg = np.array([[-1.0, -0.5, -2.0],
                         [1.0, 0.5, 2.0],
                         [0.0, 0.0, 0.0],
                         [-1.0, 0.5, 0.0]]) * np.pi
    want = np.concatenate([np.sin(want_arg), np.cos(want_arg)], axis=1)
    # sin(-pi/2) = -1, cos(pi) = -1, sin(0) = 0 ...: exact up to the rounding of pi
    exact = np.array([[0, -1, 0, -1, 0, 1],
                      [0, 1, 0, -1, 0, 1],
                      [0, 0, 0, 1, 1, 1],
                      [0, 1, 0, -1, 0, 1]], dtype=np.float64)
    assert np.allclose(want, exact, atol=1e-15)
    assert np.allclose(f, exact, atol=1e-15)
    # sine block first, then cosine block, one column per row of B
    assert f.shape == (4, 6)
