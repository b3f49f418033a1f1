"""Surrogate kernels (rsi_nn_*) on the GPU.

GEMM epilogues against a plain PyTorch FP32 reference of the same op; Adam
against the FP64 oracle; forward and backward of a small network against the
FP64 oracle MLP (oracle/mlp.py) holding the same BF16-rounded weights.
Tolerances follow from BF16 (8-bit significand, unit roundoff 2^-9 ~ 2e-3):
activations are rounded to BF16 between layers, so a few roundoffs per layer
accumulate over the network."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2408_06765_gb300 import build, rsi, surrogate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load()


def rel(a, b):
    a, b = a.double().flatten().cpu(), b.double().flatten().cpu()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (256, 512, 256), (384, 256, 96)])
def test_gemm_epilogues_match_fp32_reference(M, N, K):
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    ref = A.float() @ B.float().T
    out = torch.empty(M, N, device="cuda")
    rsi.nn_gemm("f32", A, B, out_f32=out)
    assert rel(out, ref) < 1e-5
    rsi.nn_gemm("f32", A, B, out_f32=out, bias=bias)
    assert rel(out, ref + bias) < 1e-5
    h = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    rsi.nn_gemm("bias_silu", A, B, out_f32=out, out_bf16=h, bias=bias)
    z = ref + bias
    assert rel(out, z) < 1e-5
    assert rel(h.float(), torch.nn.functional.silu(z)) < 6e-3
    aux = torch.randn(M, N, device="cuda", generator=g)
    rsi.nn_gemm("dsilu", A, B, out_bf16=h, aux=aux)
    s = torch.sigmoid(aux)
    assert rel(h.float(), ref * s * (1 + aux * (1 - s))) < 6e-3
    # split K: the same results through partial sums
    splits = K // 32
    work = torch.empty(splits * M * N, device="cuda")
    rsi.nn_gemm("f32", A, B, out_f32=out, bias=bias, splits=splits, workspace=work)
    assert rel(out, ref + bias) < 1e-5
    rsi.nn_gemm("dsilu", A, B, out_bf16=h, aux=aux, splits=splits, workspace=work)
    assert rel(h.float(), ref * s * (1 + aux * (1 - s))) < 6e-3


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 512, 256), (384, 256, 128), (256, 384, 1024),
                                   (1024, 8192, 128), (1024, 3072, 64)])
def test_gemm_tcgen05_matches_fp32_reference(M, N, K):
    """The tcgen05 engine (accumulators in tensor memory) against the same
    FP32 reference, every epilogue, with and without split K.  The engine
    takes the widest output tile that still gives every SM a tile: the small
    shapes run 64-wide tiles, 1024 x 3072 128-wide and 1024 x 8192 256-wide
    (152 SMs)."""
    g = torch.Generator(device="cuda").manual_seed(7 * M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    aux = torch.randn(M, N, device="cuda", generator=g)
    ref = A.float() @ B.float().T
    s = torch.sigmoid(aux)
    out = torch.empty(M, N, device="cuda")
    h = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    for splits in (1, K // 64):
        work = torch.empty(splits * M * N, device="cuda") if splits > 1 else None
        kw = dict(splits=splits, workspace=work, engine="tcgen05")
        out.fill_(float("nan"))
        rsi.nn_gemm("f32", A, B, out_f32=out, **kw)
        assert rel(out, ref) < 1e-5, splits
        rsi.nn_gemm("f32", A, B, out_f32=out, bias=bias, **kw)
        assert rel(out, ref + bias) < 1e-5, splits
        rsi.nn_gemm("bias_silu", A, B, out_f32=out, out_bf16=h, bias=bias, **kw)
        assert rel(out, ref + bias) < 1e-5, splits
        assert rel(h.float(), torch.nn.functional.silu(ref + bias)) < 6e-3, splits
        rsi.nn_gemm("dsilu", A, B, out_bf16=h, aux=aux, **kw)
        assert rel(h.float(), ref * s * (1 + aux * (1 - s))) < 6e-3, splits
    # both engines sum the same products in FP32: results agree closely
    o2 = torch.empty_like(out)
    rsi.nn_gemm("f32", A, B, out_f32=out, engine="tcgen05")
    rsi.nn_gemm("f32", A, B, out_f32=o2, engine="mma_sync")
    assert rel(out, o2) < 1e-6
    rsi.sync_status()  # raises if a kernel recorded a timeout


@pytest.mark.parametrize("a_t,b_t", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 512, 256), (384, 256, 192)])
def test_gemm_tcgen05_operand_layouts(M, N, K, a_t, b_t):
    """Operands read in their stored orientation: A as [K x M], B as [K x N]."""
    g = torch.Generator(device="cuda").manual_seed(3 * M + N + K + 2 * a_t + b_t)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    aux = torch.randn(M, N, device="cuda", generator=g)
    ref = A.float() @ B.float().T
    As = A.T.contiguous() if a_t else A
    Bs = B.T.contiguous() if b_t else B
    out = torch.full((M, N), float("nan"), device="cuda")
    rsi.nn_gemm("f32", As, Bs, out_f32=out, engine="tcgen05", a_t=a_t, b_t=b_t)
    assert rel(out, ref) < 1e-5
    o2 = torch.empty_like(out)
    rsi.nn_gemm("f32", A, B, out_f32=o2, engine="tcgen05")
    assert rel(out, o2) < 1e-6
    h = torch.empty(M, N, dtype=torch.bfloat16, device="cuda")
    s = torch.sigmoid(aux)
    rsi.nn_gemm("dsilu", As, Bs, out_bf16=h, aux=aux, engine="tcgen05", a_t=a_t, b_t=b_t)
    assert rel(h.float(), ref * s * (1 + aux * (1 - s))) < 6e-3
    splits = K // 64
    if splits > 1:
        work = torch.empty(splits * M * N, device="cuda")
        rsi.nn_gemm("f32", As, Bs, out_f32=out, splits=splits, workspace=work, engine="tcgen05", a_t=a_t, b_t=b_t)
        assert rel(out, ref) < 1e-5
    rsi.sync_status()


def test_gemm_layout_needs_tcgen05():
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    out = torch.empty(128, 128, device="cuda")
    with pytest.raises(rsi.RSIError):
        rsi.nn_gemm("f32", A.T.contiguous(), torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda"),
                    out_f32=out, engine="mma_sync", a_t=True)


def test_transpose_colsum_cast():
    x = torch.randn(300, 70, device="cuda").to(torch.bfloat16)
    t = torch.empty(70, 300, dtype=torch.bfloat16, device="cuda")
    rsi.nn_transpose(x, t)
    assert torch.equal(t, x.T)
    cs = torch.empty(70, device="cuda")
    rsi.nn_colsum(x, cs)
    assert rel(cs, x.float().sum(0)) < 1e-5
    f = torch.randn(1000, device="cuda")
    h = torch.empty(1000, dtype=torch.bfloat16, device="cuda")
    rsi.nn_cast_bf16(f, h)
    assert torch.equal(h, f.to(torch.bfloat16))


@pytest.mark.parametrize("n", [4096, 4099])  # four elements per thread; a ragged count takes the scalar kernel
def test_adam_matches_oracle(n):
    rng = np.random.default_rng(0)
    w0 = rng.normal(size=n)
    w = torch.tensor(w0, dtype=torch.float32, device="cuda")
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    wh = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    wo, mo, vo = w0.astype(np.float32).astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        g = rng.normal(size=n)
        rsi.nn_adam(w, m, v, torch.tensor(g, dtype=torch.float32, device="cuda"), 1e-3, step, w_bf16=wh)
        wo, mo, vo = omlp.adam_step(wo, g.astype(np.float32).astype(np.float64), mo, vo, step, 1e-3)
    assert np.max(np.abs(w.cpu().numpy() - wo)) < 1e-6
    assert torch.equal(wh, w.to(torch.bfloat16))  # the bf16 copy is the rounded master weight


def test_carrier_coeffs_on_device():
    """rsi_nn_carrier_coeffs against the same definition in numpy (FP64), on
    300 rows that include post-critical tilts, and the f32 inputs."""
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * np.random.default_rng(2).uniform(size=(300, 5))
    p64 = torch.tensor(params, dtype=torch.float64, device="cuda")
    car = torch.empty(300, 4, dtype=torch.float64, device="cuda")
    p32 = torch.empty(300, 5, dtype=torch.float32, device="cuda")
    rsi.nn_carrier_coeffs(p64, surrogate.C1, surrogate.C2, car, p32)
    assert np.allclose(car.cpu().numpy(), surrogate.carrier_coeffs(params), rtol=1e-13, atol=1e-9)
    assert torch.equal(p32.cpu(), torch.tensor(params, dtype=torch.float32))


def test_carrier_round_trip_and_definition():
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * np.random.default_rng(1).uniform(size=(3, 5))
    img = torch.randn(3, 128, 128, dtype=torch.complex64, device="cuda")
    env = surrogate.demodulate(img, params)
    back = surrogate.modulate(env, params)
    assert rel(torch.view_as_real(back), torch.view_as_real(img)) < 1e-6
    # the amplitude scale rides along in the same pass
    back3 = surrogate.modulate(env, params, scale=3.0)
    assert rel(torch.view_as_real(back3), 3.0 * torch.view_as_real(back)) < 1e-6
    # psi at one pixel, restated
    x_off, tilt, path, f, depth = params[0]
    k1, k2 = 2 * np.pi * f / 1480.0, 2 * np.pi * f / 5900.0
    s = 5900.0 / 1480.0 * np.sin(tilt)
    c = np.sqrt(max(0.0, 1 - s * s))
    x = -20e-3 + (5 + 0.5) * 40e-3 / 128
    z = 0.0 + (7 + 0.5) * 40e-3 / 128
    psi = k1 * path + k2 * (s * x + c * (z + depth))
    want = complex(img[0, 7, 5]) * np.exp(-1j * psi)
    got = env[0].view(128, 128, 2)[7, 5]
    assert abs(complex(got[0], got[1]) - want) < 1e-5 * abs(want) + 1e-6
    # every pixel of every image against the same definition in FP64
    xs = -20e-3 + (np.arange(128) + 0.5) * 40e-3 / 128
    zs = (np.arange(128) + 0.5) * 40e-3 / 128
    full = img.cpu().numpy().astype(np.complex128)
    for b in range(3):
        x_off, tilt, path, f, depth = params[b]
        k1, k2 = 2 * np.pi * f / 1480.0, 2 * np.pi * f / 5900.0
        s = 5900.0 / 1480.0 * np.sin(tilt)
        c = np.sqrt(max(0.0, 1 - s * s))
        psi = k1 * path + k2 * (s * xs[None, :] + c * (zs[:, None] + depth))
        want = full[b] * np.exp(-1j * psi)
        e = env[b].view(128, 128, 2).cpu().numpy().astype(np.float64)
        got = e[..., 0] + 1j * e[..., 1]
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-5, b


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_graphed_inference_matches_eager(engine):
    """The CUDA-graph inference path gives the eager path's images, on two
    batches in a row (its pinned staging buffers are reused).  With the
    tcgen05 engine the output layer applies the carrier in the GEMM
    epilogue, advancing the phase by rotation within blocks of 16 pixels
    (about 1e-6 from the per-pixel phase of the separate carrier pass); with
    mma.sync the graph holds the separate pass."""
    net = surrogate.MLP(batch=256, seed=5, engine=engine)
    g = surrogate.GraphedInference(net, scale=0.7)
    rng = np.random.default_rng(9)
    for _ in range(2):
        params = surrogate.LO + (surrogate.HI - surrogate.LO) * rng.uniform(size=(256, 5))
        got = g(params).clone()
        pq = torch.tensor(params, dtype=torch.float32, device="cuda")
        want = surrogate.modulate(net.predict(pq), params, scale=0.7)
        assert rel(torch.view_as_real(got), torch.view_as_real(want)) < 1e-5
    rsi.sync_status()


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_graphed_training_matches_eager(engine):
    """Training through the CUDA graph (GraphedTrainer: batch gathered into
    fixed buffers, Adam's schedule read from the device) takes the same steps
    as eager training: same losses, same weights after two epochs."""
    rng = np.random.default_rng(11)
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * rng.uniform(size=(512, 5))
    env = torch.tensor(rng.normal(size=(512, 256)) * 0.5, dtype=torch.float32, device="cuda")
    nets = [small_net(engine), small_net(engine)]
    losses = [surrogate.train(net, params, env, epochs=2, lr=3e-3, graph=g) for net, g in zip(nets, (False, True))]
    assert nets[0].step_count == nets[1].step_count == 8
    assert np.allclose(losses[0], losses[1], rtol=1e-5, atol=0)
    for a, b in zip(nets[0].W + nets[0].b, nets[1].W + nets[1].b):
        assert rel(b, a) < 1e-5
    rsi.sync_status()


@pytest.mark.parametrize("M,K", [(256, 512), (128, 64)])
def test_gemm_carrier_matches_gemm_then_carrier(M, K):
    """The fused output layer + carrier (rsi_nn_gemm_carrier) against the GEMM
    followed by the carrier pass, and against the carrier's FP64 definition
    on every pixel of two images."""
    g = torch.Generator(device="cuda").manual_seed(M + K)
    N = 2 * 128 * 128
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = (torch.randn(N, K, device="cuda", generator=g) / K ** 0.5).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * np.random.default_rng(M).uniform(size=(M, 5))
    car = torch.tensor(surrogate.carrier_coeffs(params), dtype=torch.float64, device="cuda")
    y = torch.empty(M, N, device="cuda")
    rsi.nn_gemm("f32", A, B, out_f32=y, bias=bias, engine="tcgen05")
    want = torch.empty_like(y)
    rsi.nn_carrier(car, surrogate.WINDOW, +1, y, want, scale=1.5)
    got = torch.full_like(y, float("nan"))
    rsi.nn_gemm_carrier(A, B, bias, car, surrogate.WINDOW, +1, 1.5, got)
    rsi.sync_status()
    assert rel(got, want) < 1e-5
    yc = y.double().cpu().numpy()
    xs = -20e-3 + (np.arange(128) + 0.5) * 40e-3 / 128
    zs = (np.arange(128) + 0.5) * 40e-3 / 128
    c = surrogate.carrier_coeffs(params)
    for b in (0, M - 1):
        psi = c[b, 0] * xs[None, :] + c[b, 1] * zs[:, None] + c[b, 2]
        ref = 1.5 * (yc[b, 0::2] + 1j * yc[b, 1::2]).reshape(128, 128) * np.exp(1j * psi)
        gb = got[b].double().cpu().numpy()
        out = (gb[0::2] + 1j * gb[1::2]).reshape(128, 128)
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-5, b
    with pytest.raises(rsi.RSIError):  # N must match the window
        rsi.nn_gemm_carrier(A, B[:N // 2], bias, car, surrogate.WINDOW, +1, 1.0, got[:, :N // 2])


def test_gemm_carrier_row_wrap_and_sign():
    """A window of 24 x 8 pixels (N = 384): image rows end inside blocks of 16
    pixels, where the fused epilogue restarts from the exact phase; sign -1
    (demodulation)."""
    g = torch.Generator(device="cuda").manual_seed(5)
    M, K, nx, nz = 128, 64, 24, 8
    N = 2 * nx * nz
    win = {"x0": -3e-3, "x1": 4e-3, "nx": nx, "z0": 1e-3, "z1": 9e-3, "nz": nz}
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = (torch.randn(N, K, device="cuda", generator=g) / K ** 0.5).to(torch.bfloat16)
    bias = torch.randn(N, device="cuda", generator=g)
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * np.random.default_rng(6).uniform(size=(M, 5))
    car = torch.tensor(surrogate.carrier_coeffs(params), dtype=torch.float64, device="cuda")
    y = torch.empty(M, N, device="cuda")
    rsi.nn_gemm("f32", A, B, out_f32=y, bias=bias, engine="tcgen05")
    want = torch.empty_like(y)
    rsi.nn_carrier(car, win, -1, y, want, scale=0.5)
    got = torch.full_like(y, float("nan"))
    rsi.nn_gemm_carrier(A, B, bias, car, win, -1, 0.5, got)
    rsi.sync_status()
    assert rel(got, want) < 1e-5


def small_net(engine="tcgen05"):
    return surrogate.MLP(n_freq=64, width=128, depth=2, n_out=256, batch=128, seed=3, sigma_b=1.0, engine=engine)


def oracle_params(net):
    Wq = [w16.double().cpu().numpy() for w16 in net.W16]  # the BF16 weights the GPU multiplies by
    bq = [b.double().cpu().numpy() for b in net.b]
    return {"W": Wq, "b": bq}


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync"])
def test_forward_backward_match_fp64_oracle(engine):
    net = small_net(engine)
    rng = np.random.default_rng(4)
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * rng.uniform(size=(128, 5))
    t = rng.normal(size=(128, 256)) * 0.5
    p_d = torch.tensor(params, dtype=torch.float32, device="cuda")
    t_d = torch.tensor(t, dtype=torch.float32, device="cuda")
    y = net.forward(p_d).clone()
    loss = float(net.loss(t_d).item())
    net.backward()
    torch.cuda.synchronize()
    P = oracle_params(net)
    p32 = params.astype(np.float32).astype(np.float64)
    yo, cache = omlp.forward(P, p32, surrogate.LO.astype(np.float32), surrogate.HI.astype(np.float32),
                             net.fmat.double().cpu().numpy())
    go = omlp.backward(P, cache, yo, t)
    assert rel(y, torch.tensor(yo)) < 2e-2
    assert abs(loss - omlp.loss(yo, t)) < 2e-2 * omlp.loss(yo, t)
    for l in range(len(P["W"])):
        assert rel(net.gW[l], torch.tensor(go["W"][l])) < 5e-2, l
        assert rel(net.gb[l], torch.tensor(go["b"][l])) < 5e-2, l


def test_training_reduces_the_loss():
    net = small_net()
    rng = np.random.default_rng(5)
    params = surrogate.LO + (surrogate.HI - surrogate.LO) * rng.uniform(size=(1024, 5))
    u = 2 * (params - surrogate.LO) / (surrogate.HI - surrogate.LO) - 1
    t = np.sin(np.pi * u @ rng.normal(size=(5, 256)) * 0.5)  # smooth target family
    env = torch.tensor(t, dtype=torch.float32, device="cuda")
    losses = surrogate.train(net, params, env, epochs=100, lr=3e-3)
    assert losses[-1] < 0.25 * losses[0]


@pytest.mark.slow
def test_surrogate_pipeline_gain_and_gate():
    """Train on fields from the batched RSI path (reduced counts), measure the
    held-out error, the inference rate against the RSI path, and that the gate
    sends queries whose error estimate exceeds 1e-2 back to the RSI path."""
    import time
    from paper_2408_06765_gb300 import workloads as W
    n = 1536
    params = W.c5_params(n, seed=1)
    t0 = time.perf_counter()
    imgs = surrogate.rsi_images(params, n_piston=1 << 12, n_iface=1 << 14)
    torch.cuda.synchronize()
    rsi_rate = n / (time.perf_counter() - t0)
    env = surrogate.demodulate(imgs, params)
    tr, ho = slice(0, 1280), slice(1280, 1536)
    scale = float(env[tr].pow(2).mean().sqrt())
    net = surrogate.MLP(batch=256)
    net.scale = scale
    losses = surrogate.train(net, params[tr], env[tr] / scale, epochs=20, lr=1e-3)
    assert losses[-1] < losses[0]
    pb = torch.tensor(params[ho], dtype=torch.float32, device="cuda")
    pred = surrogate.modulate(net.predict(pb), params[ho], scale=scale)
    errs = surrogate.rel_errors(pred, imgs[ho]).cpu().numpy()
    assert np.all(np.isfinite(errs))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        surrogate.modulate(net.predict(pb), params[ho], scale=scale)
    torch.cuda.synchronize()
    nn_rate = 5 * 256 / (time.perf_counter() - t0)
    assert nn_rate > rsi_rate  # what the network gains over the method
    sur = surrogate.Surrogate(net, params[ho], errs, threshold=1e-2)
    q = params[:256]
    img, est, fall = sur.infer(q)
    assert set(fall.tolist()) == set(np.nonzero(est > 1e-2)[0].tolist())
    if len(fall):
        ref = surrogate.rsi_images(q[fall], index0=10**6)
        assert torch.equal(img[torch.tensor(fall, device="cuda")], ref)
