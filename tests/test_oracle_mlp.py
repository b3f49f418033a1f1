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
