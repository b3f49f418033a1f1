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




# ---------------------------------------------------------------------------
# the coordinate network (rsi_nn_rows / forward / backward / targets / infer)
# against its FP64 oracle (oracle/coordnet.py)
# ---------------------------------------------------------------------------
# BF16 carries 8 significant bits (unit roundoff u = 2^-9 ~ 2e-3).  The row
# inputs c are formed in FP32 (a few roundings and FP32 transcendentals: about
# 1e-6 absolute each) and each network input is rounded once to BF16, so an
# input differs from the oracle's FP64 value by at most half a BF16 ulp
# (<= 2^-8 |v|) plus its FP32 error: 1e-5 for c itself, pi sum_k |B_fk| 1e-6
# for a Fourier feature (the error of its argument).  The forward
# rounds each hidden layer's output to BF16 once (FP32 accumulation within a
# GEMM), so with the same BF16 inputs and weights the head outputs differ by a
# few u: relative L2 <= 1e-2 for two hidden layers.  The backward adds one
# BF16 rounding of dZ per layer: gradients within 2e-2 relative L2 per layer,
# and the gradient's norm within 1e-3 (the roundings are unbiased, so the
# norm's error is second order).
from oracle import coordnet as ocn  # noqa: E402
import oracle as orc  # noqa: E402


def small_coordnet(rows=16384, F=56, W=128, D=2, seed=3):
    return surrogate.CoordNet(n_freq=F, width=W, depth=D, rows=rows, seed=seed)


def act_view(net, what):
    """Views into the activation workspace, at the offsets of nn_net.cu's layout."""
    R, K0, Wd, D = net.rows, 2 * net.n_freq + 16, net.width, net.depth
    off = 0
    out = {}

    def take(key, nbytes):
        nonlocal off
        out[key] = off
        off = (off + nbytes + 255) // 256 * 256

    take("h0", R * K0 * 2)
    for l in range(1, D + 1):
        take(f"z{l}", R * Wd * 4)
        take(f"h{l}", R * Wd * 2)
    take("y", R * 16)
    take("t", R * 16)
    o = out[what]
    if what == "h0":
        return net.act[o:o + R * K0 * 2].view(torch.bfloat16).view(R, K0)
    if what in ("y", "t"):
        return net.act[o:o + R * 16].view(torch.float32).view(R, 4)
    return net.act[o:o + R * Wd * 2].view(torch.bfloat16).view(R, Wd)


def field_params(n, seed=0):
    rng = np.random.default_rng(seed)
    p = surrogate.LO + (surrogate.HI - surrogate.LO) * rng.uniform(size=(n, 5))
    p[0, 1] = -abs(p[0, 1])                       # a negative tilt (mirrored inputs)
    p[1, 1] = surrogate.CRIT + 0.02               # past the critical angle
    p[2, 1] = 0.0
    return p


def row_tolerance(net, want):
    """Per-value bound of a GPU input row against the oracle's (see above)."""
    B = net.fmat.cpu().numpy().astype(np.float64)
    arg_err = np.pi * np.abs(B).sum(axis=1) * 1e-6
    extra = np.concatenate([arg_err, arg_err, np.full(16, 1e-5)])
    return 2.0 ** -8 * np.abs(want) + extra[None, :]


def oracle_rows(net, params, b, q):
    c = ocn.row_inputs(params[b], q % 128, q // 128, surrogate.WINDOW, surrogate.BOX_LO, surrogate.BOX_HI,
                       surrogate.C1, surrogate.C2, surrogate.A_PISTON)
    return ocn.features(c, net.fmat.cpu().numpy().astype(np.float64))


def test_coordnet_rows_match_oracle():
    net = small_coordnet()
    params = field_params(6)
    p64 = torch.tensor(params, device="cuda")
    n = params.shape[0]
    rng = np.random.default_rng(1)
    tg = torch.tensor(rng.normal(size=(n, surrogate.NPIX * 2)), dtype=torch.float32, device="cuda")
    lr = torch.tensor(rng.normal(size=n), dtype=torch.float32, device="cuda")
    # PIXELS mode from a ragged first row: field-major pairs
    first = 3 * surrogate.NPIX + 777
    rsi.nn_rows(net.net, p64, n, "pixels", net.act, first=first, targets=tg, log_rms=lr)
    torch.cuda.synchronize()
    g = np.arange(net.rows) + first
    g = np.minimum(g, n * surrogate.NPIX - 1)
    b, q = g // surrogate.NPIX, g % surrogate.NPIX
    sel = rng.choice(net.rows, 3000, replace=False)
    want = oracle_rows(net, params, b[sel], q[sel])
    got = act_view(net, "h0")[torch.tensor(sel, device="cuda")].float().cpu().numpy()
    excess = np.abs(got - want) - row_tolerance(net, want)
    assert np.all(excess <= 0), (excess.max(), np.unravel_index(excess.argmax(), excess.shape))
    tr = act_view(net, "t").cpu().numpy()[sel]
    tgn = tg.view(n, -1, 2).cpu().numpy()
    assert np.array_equal(tr[:, 0], tgn[b[sel], q[sel], 0]) and np.array_equal(tr[:, 1], tgn[b[sel], q[sel], 1])
    assert np.array_equal(tr[:, 2], lr.cpu().numpy()[b[sel]]) and np.all(tr[:, 3] == 0)
    # RANDOM mode: the pair of row r from SplitMix64 at seed + (r + 1) gamma
    seed = 123456789
    rsi.nn_rows(net.net, p64, n, "random", net.act, seed=seed, targets=tg, log_rms=lr)
    torch.cuda.synchronize()
    gamma = 0x9E3779B97F4A7C15
    sel = rng.choice(net.rows, 500, replace=False)
    u = np.array([orc.mix64((seed + gamma * (int(r) + 1)) % 2**64) for r in sel], dtype=np.uint64)
    b = ((u >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    q = ((u & np.uint64(0xFFFFFFFF)) * np.uint64(surrogate.NPIX)) >> np.uint64(32)
    b, q = b.astype(np.int64), q.astype(np.int64)
    want = oracle_rows(net, params, b, q)
    got = act_view(net, "h0")[torch.tensor(sel, device="cuda")].float().cpu().numpy()
    excess = np.abs(got - want) - row_tolerance(net, want)
    assert np.all(excess <= 0), (excess.max(), np.unravel_index(excess.argmax(), excess.shape))
    tr = act_view(net, "t").cpu().numpy()[sel]
    assert np.array_equal(tr[:, 0], tgn[b, q, 0]) and np.array_equal(tr[:, 2], lr.cpu().numpy()[b])


def oracle_params(net):
    """The network's weights as the GPU uses them: hidden W in BF16, biases
    and the head in FP32."""
    Ws, bs = [], []
    for l in range(net.depth + 1):
        W = net.layer(l)
        Ws.append((W.to(torch.bfloat16) if l < net.depth else W).double().cpu().numpy())
        bs.append(net.layer(l, bias=True).double().cpu().numpy())
    return {"W": Ws, "b": bs}


def test_coordnet_forward_backward_match_oracle():
    net = small_coordnet(rows=1024)
    params = field_params(4, seed=5)
    p64 = torch.tensor(params, device="cuda")
    rng = np.random.default_rng(2)
    tg = torch.tensor(rng.normal(size=(4, surrogate.NPIX * 2)) * 0.5, dtype=torch.float32, device="cuda")
    lr = torch.tensor(rng.normal(size=4), dtype=torch.float32, device="cuda")
    rsi.nn_rows(net.net, p64, 4, "random", net.act, seed=77, targets=tg, log_rms=lr)
    y = net.forward().clone()
    loss = float(net.backward().item())
    torch.cuda.synchronize()
    rsi.sync_status()
    h0 = act_view(net, "h0").double().cpu().numpy()
    t = act_view(net, "t").double().cpu().numpy()[:, :3]
    P = oracle_params(net)
    yo, cache = ocn.forward(P, h0)
    go = ocn.backward(P, cache, yo, t)
    assert np.all(y.cpu().numpy()[:, 3] == 0)
    assert rel(y[:, :3], torch.tensor(yo)) < 1e-2
    assert abs(loss - ocn.loss(yo, t)) < 2e-2 * ocn.loss(yo, t)
    gn2, gon2 = 0.0, 0.0
    for l in range(net.depth + 1):
        gW, gb = net.layer(l, buf=net.g), net.layer(l, bias=True, buf=net.g)
        assert rel(gW, torch.tensor(go["W"][l])) < 2e-2, l
        assert rel(gb, torch.tensor(go["b"][l])) < 2e-2, l
        gn2 += float(gW.double().pow(2).sum() + gb.double().pow(2).sum())
        gon2 += float((go["W"][l] ** 2).sum() + (go["b"][l] ** 2).sum())
    assert abs(math.sqrt(gn2) / math.sqrt(gon2) - 1.0) < 1e-3


def test_coordnet_targets_and_infer_match_definitions():
    net = small_coordnet()
    params = field_params(3, seed=7)
    p64 = torch.tensor(params, device="cuda")
    g = torch.Generator(device="cuda").manual_seed(9)
    img = torch.randn(3, 128, 128, dtype=torch.complex64, device="cuda", generator=g)
    ts = surrogate.TrainingSet(net, params, img)
    torch.cuda.synchronize()
    # targets: image times exp(-i psi) over its RMS, and the log RMS (FP64 restatement)
    car = surrogate.carrier_coeffs(params)
    xs = -20e-3 + (np.arange(128) + 0.5) * 40e-3 / 128
    zs = (np.arange(128) + 0.5) * 40e-3 / 128
    full = img.cpu().numpy().astype(np.complex128)
    tgt = ts.targets.view(3, 128, 128, 2).double().cpu().numpy()
    for bq in range(3):
        psi = car[bq, 0] * xs[None, :] + car[bq, 1] * zs[:, None] + car[bq, 2]
        env = full[bq] * np.exp(-1j * psi)
        rms = np.sqrt(np.mean(np.abs(env) ** 2))
        got = tgt[bq, ..., 0] + 1j * tgt[bq, ..., 1]
        assert np.linalg.norm(got - env / rms) / np.linalg.norm(env / rms) < 1e-5
        assert abs(float(ts.log_rms[bq]) - math.log(rms)) < 1e-5
    # infer: rows through the network, then the oracle's image assembly of the
    # same head outputs (3 fields, rows of one field per call)
    out = net.infer(p64)
    torch.cuda.synchronize()
    rsi.sync_status()
    P = oracle_params(net)
    for bq in range(3):
        q = np.arange(surrogate.NPIX)
        h0 = oracle_rows(net, params, np.full(q.size, bq), q)
        yo, _ = ocn.forward(P, h0)
        want = ocn.image(yo, params[bq], surrogate.WINDOW, surrogate.C1, surrogate.C2)
        got = out[bq].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 2e-2, bq


def test_coordnet_graphed_training_matches_eager():
    params = field_params(8, seed=11)
    g = torch.Generator(device="cuda").manual_seed(3)
    img = torch.randn(8, 128, 128, dtype=torch.complex64, device="cuda", generator=g)
    nets = [small_coordnet(rows=2048, seed=4) for _ in range(2)]
    for net, graph in zip(nets, (False, True)):
        ts = surrogate.TrainingSet(net, params, img)
        surrogate.train(net, ts, steps=6, lr=1e-3, warmup=2, graph=graph, seed=5)
    torch.cuda.synchronize()
    # the same kernels on the same rows: bit-identical weights
    assert torch.equal(nets[0].w, nets[1].w)
    assert nets[0].step_count == nets[1].step_count == 6


@pytest.mark.slow
def test_surrogate_gate_serves_accurate_fields_faster_than_rsi():
    """What the trained network gains over the plain RSI path: on a sub-box
    of the c5 inputs (tilt up to 5 degrees, 2-4 MHz, the full water-path,
    depth and offset ranges), trained on 2048 RSI fields for 40 000 steps,
    the gate (mean held-out error of the 8 nearest held-out fields <= 1e-2)
    serves at least half of the queries, the fields it serves are within 1e-2
    of the RSI path (median; each within 3e-2), and the network delivers them
    at least 20 times faster than the RSI path computes them."""
    import time
    gen = np.random.Generator(np.random.Philox(key=99))
    lo = np.array([-10e-3, 0.0, 20e-3, 2e6, 1e-3])
    hi = np.array([10e-3, math.radians(5.0), 60e-3, 4e6, 20e-3])
    params = lo + (hi - lo) * gen.random((2560, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    imgs = surrogate.rsi_images(params)
    torch.cuda.synchronize()
    rsi_fields_s = len(params) / (time.perf_counter() - t0)
    ntr = 2048
    net = surrogate.CoordNet(rows=32768)
    ts = surrogate.TrainingSet(net, params[:ntr], imgs[:ntr])
    surrogate.train(net, ts, steps=40000, lr=1e-3)
    held = torch.tensor(params[ntr:], device="cuda")
    out = torch.empty(len(held), surrogate.NPIX * 2, dtype=torch.float32, device="cuda")
    net.infer(held, out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pred = net.infer(held, out)
    torch.cuda.synchronize()
    nn_fields_s = len(held) / (time.perf_counter() - t0)
    rsi.sync_status()
    errs = surrogate.rel_errors(pred, imgs[ntr:]).cpu().numpy()
    sur = surrogate.Surrogate(net, params[ntr:ntr + 256], errs[:256], threshold=1e-2)
    est = sur.error_estimate(params[ntr + 256:])
    served = est <= 1e-2
    assert served.mean() >= 0.5, served.mean()
    assert np.median(errs[256:][served]) <= 1e-2
    assert errs[256:][served].max() <= 3e-2
    assert nn_fields_s >= 20 * rsi_fields_s, (nn_fields_s, rsi_fields_s)
    # the gate's images: the network's where it serves, the RSI path's (other
    # QMC point sets, so within the QMC noise) where it does not; a strict
    # threshold sends some queries back
    q = params[ntr + 256:ntr + 288]
    strict = surrogate.Surrogate(net, params[ntr:ntr + 256], errs[:256], threshold=float(np.median(est)))
    img, est_q, fall = strict.infer(q)
    assert 0 < len(fall) < len(q)
    got = surrogate.rel_errors(img, imgs[ntr + 256:ntr + 288]).cpu().numpy()
    assert np.all(got[fall] <= 2e-2) and np.median(got) <= 1e-2
