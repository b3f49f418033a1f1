"""Learned surrogate of the RSI chain (not in the paper): a Fourier-feature MLP
that maps (x-offset, tilt, water path, frequency, image depth) to the
128 x 128 field image of one water -> steel chain, trained on images the GPU
RSI path computes, with the RSI path as its fallback and the measure of its error.

Every numerical step runs in librsi.so (rsi_nn_* kernels: BF16 tensor-core
GEMMs with FP32 accumulation and fused bias/SiLU epilogues, FP32 master
weights, Adam); this module sequences the calls and keeps the buffers.

Network (same definition as the FP64 oracle, oracle/mlp.py):
    u = 2 (p - lo)/(hi - lo) - 1;  h0 = [sin(pi B u), cos(pi B u)]
    h_l = silu(W_l h_{l-1} + b_l), l = 1..depth;  y = W_out h_depth + b_out
The output y is the image times exp(-i psi), psi the phase of the refracted
plane wave: psi = k1 L + k2 (s x + c (z + depth)) with L the water path,
s = (c2/c1) sin(tilt) and c = sqrt(1 - s^2) (0 past the critical angle), x, z
measured from the point where the axis meets the interface and from the
window's top edge; real and imaginary parts interleaved and divided by a
fixed amplitude scale.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import rsi
from . import workloads as W

C1, C2 = W.WATER["c"], W.STEEL["c"]
LO = np.array([-10e-3, math.radians(-15.0), 20e-3, 2e6, 1e-3])
HI = np.array([10e-3, math.radians(15.0), 60e-3, 10e6, 20e-3])
WINDOW = {"x0": -20e-3, "x1": 20e-3, "nx": 128, "z0": 0.0, "z1": 40e-3, "nz": 128}


def carrier_coeffs(params) -> np.ndarray:
    """(kx, kz, phi0, 0) per sample: psi = kx x + kz z + phi0 is the phase of
    the refracted plane wave (water path phase k1 L included)."""
    p = np.atleast_2d(np.asarray(params, np.float64))
    k1 = 2 * np.pi * p[:, 3] / C1
    k2 = 2 * np.pi * p[:, 3] / C2
    s = C2 / C1 * np.sin(p[:, 1])
    c = np.sqrt(np.clip(1.0 - s * s, 0.0, None))
    return np.stack([k2 * s, k2 * c, k1 * p[:, 2] + k2 * c * p[:, 4], np.zeros(len(p))], axis=1)


class MLP:
    """Weights, Adam state and activation buffers of the surrogate."""

    def __init__(self, n_freq=128, width=512, depth=4, n_out=2 * 128 * 128, batch=256, seed=0,
                 sigma_b=2.0, device="cuda", engine="tcgen05"):
        self.n_in, self.F, self.width, self.depth, self.n_out = 5, n_freq, width, depth, n_out
        self.batch = batch
        self.engine = engine  # GEMM engine: "tcgen05" (tensor memory) or "mma_sync"
        self.device = device
        rng = np.random.default_rng(seed)
        dims = [2 * n_freq] + [width] * depth + [n_out]
        self.dims = dims
        f32 = dict(dtype=torch.float32, device=device)
        # Every weight and bias (and its moments, gradient and bf16 copy) is a
        # view into one flat buffer per role, segments padded to 64 elements
        # (128-byte aligned for the GEMMs' tensor maps), so that one Adam
        # launch updates all parameters; padding has zero gradient and stays 0.
        pad = lambda n: (n + 63) // 64 * 64
        shapes = [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]
        total = sum(pad(r * c) + pad(r) for r, c in shapes)
        self.flat = {k: torch.zeros(total, **f32) for k in ("w", "m", "v", "g")}
        self.flat16 = torch.zeros(total, dtype=torch.bfloat16, device=device)
        views = {k: ([], []) for k in ("w", "m", "v", "g", "h")}
        off = 0
        for r, c in shapes:
            for k in ("w", "m", "v", "g", "h"):
                buf = self.flat16 if k == "h" else self.flat[k]
                views[k][0].append(buf[off:off + r * c].view(r, c))
                views[k][1].append(buf[off + pad(r * c):off + pad(r * c) + r])
            off += pad(r * c) + pad(r)
        self.W, self.b = views["w"]
        self.mW, self.mb = views["m"]
        self.vW, self.vb = views["v"]
        self.gW, self.gb = views["g"]
        self.W16 = views["h"][0]
        for i, (r, c) in enumerate(shapes):
            std = math.sqrt(2.0 / dims[i]) if i < len(dims) - 2 else math.sqrt(1.0 / dims[i])
            self.W[i].copy_(torch.tensor(rng.normal(0.0, std, size=(r, c)), **f32))
        self.fmat = torch.tensor(rng.normal(0.0, sigma_b, size=(n_freq, 5)), **f32)
        self.lo = torch.tensor(LO, **f32)
        self.hi = torch.tensor(HI, **f32)
        rsi.nn_cast_bf16(self.flat["w"], self.flat16)
        self.step_count = 0
        self.scale = 1.0
        self._alloc(batch)

    def _alloc(self, B):
        d, bf = self.device, torch.bfloat16
        self.B_alloc = B
        self.H = [torch.empty((B, n), dtype=bf, device=d) for n in self.dims[:-1]]
        self.Z = [torch.empty((B, n), dtype=torch.float32, device=d) for n in self.dims[1:-1]]
        self.y = torch.empty((B, self.n_out), dtype=torch.float32, device=d)
        self.dy = torch.empty((B, self.n_out), dtype=bf, device=d)
        self.dZ = [torch.empty((B, n), dtype=bf, device=d) for n in self.dims[1:-1]]
        self.HT = [torch.empty((n, B), dtype=bf, device=d) for n in self.dims[:-1]]
        self.dyT = torch.empty((self.n_out, B), dtype=bf, device=d)
        self.dZT = [torch.empty((n, B), dtype=bf, device=d) for n in self.dims[1:-1]]
        self.WT = [torch.empty((w.shape[1], w.shape[0]), dtype=bf, device=d) for w in self.W]
        self.partial = torch.empty(1024, dtype=torch.float64, device=d)
        # split K for the backward GEMM through the output layer (few output
        # tiles, K = n_out): about one (tcgen05, persistent) or two (mma.sync)
        # CTAs per SM
        if self.engine == "tcgen05":
            tiles = (B // 128) * (self.width // (256 if self.width % 256 == 0 else 128))
            self.splits_out = max(1, min(self.n_out // 64, 152 // max(1, tiles)))
        else:
            tiles = (B // 128) * (self.width // 128)
            self.splits_out = max(1, min(self.n_out // 32, (2 * 152) // max(1, tiles)))
        self.work = torch.empty(self.splits_out * B * self.width if self.splits_out > 1 else 1,
                                dtype=torch.float32, device=d)
        self.loss_buf = torch.empty(1, dtype=torch.float32, device=d)

    # -- forward / backward / update ------------------------------------------
    def hidden(self, p) -> torch.Tensor:
        """Features and hidden layers: the last hidden activations (bf16)."""
        assert p.shape[0] == self.B_alloc
        rsi.nn_features(p, self.lo, self.hi, self.fmat, self.H[0])
        for l in range(self.depth):
            rsi.nn_gemm("bias_silu", self.H[l], self.W16[l], out_f32=self.Z[l], out_bf16=self.H[l + 1],
                        bias=self.b[l], engine=self.engine)
        return self.H[self.depth]

    def forward(self, p) -> torch.Tensor:
        """p: f32 [B, 5] on the device (B = the allocated batch)."""
        self.hidden(p)
        rsi.nn_gemm("f32", self.H[self.depth], self.W16[-1], out_f32=self.y, bias=self.b[-1], engine=self.engine)
        return self.y

    def loss(self, t, grad: bool = True) -> torch.Tensor:
        n = self.y.numel()
        rsi.nn_loss(self.y, t, 2.0 / n, self.dy if grad else None, self.partial, self.loss_buf)
        return self.loss_buf

    def backward(self):
        """Gradients of the mean squared error into gW, gb (after loss())."""
        L = self.depth
        tc = self.engine == "tcgen05"
        # gW[L] = dy^T H[L]; dZ[L-1] = (dy W[L]) * silu'(Z[L-1]).  The tcgen05
        # engine reads the stored matrices in either orientation; the mma.sync
        # engine needs K-contiguous copies.
        if tc:
            rsi.nn_gemm("f32", self.dy, self.H[L], out_f32=self.gW[L], engine="tcgen05", a_t=True, b_t=True)
        else:
            rsi.nn_transpose(self.dy, self.dyT)
            rsi.nn_transpose(self.H[L], self.HT[L])
            rsi.nn_gemm("f32", self.dyT, self.HT[L], out_f32=self.gW[L], engine=self.engine)
        rsi.nn_colsum(self.dy, self.gb[L])
        if tc:
            rsi.nn_gemm("dsilu", self.dy, self.W16[L], out_bf16=self.dZ[L - 1], aux=self.Z[L - 1],
                        splits=self.splits_out, workspace=self.work, engine="tcgen05", b_t=True)
        else:
            rsi.nn_transpose(self.W16[L], self.WT[L])
            rsi.nn_gemm("dsilu", self.dy, self.WT[L], out_bf16=self.dZ[L - 1], aux=self.Z[L - 1],
                        splits=self.splits_out, workspace=self.work, engine=self.engine)
        for l in range(L - 1, -1, -1):
            if tc:
                rsi.nn_gemm("f32", self.dZ[l], self.H[l], out_f32=self.gW[l], engine="tcgen05", a_t=True, b_t=True)
            else:
                rsi.nn_transpose(self.dZ[l], self.dZT[l])
                rsi.nn_transpose(self.H[l], self.HT[l])
                rsi.nn_gemm("f32", self.dZT[l], self.HT[l], out_f32=self.gW[l], engine=self.engine)
            rsi.nn_colsum(self.dZ[l], self.gb[l])
            if l > 0:
                if tc:
                    rsi.nn_gemm("dsilu", self.dZ[l], self.W16[l], out_bf16=self.dZ[l - 1], aux=self.Z[l - 1],
                                engine="tcgen05", b_t=True)
                else:
                    rsi.nn_transpose(self.W16[l], self.WT[l])
                    rsi.nn_gemm("dsilu", self.dZ[l], self.WT[l], out_bf16=self.dZ[l - 1], aux=self.Z[l - 1],
                                engine=self.engine)

    def adam(self, lr: float):
        """One Adam step on every parameter: a single launch over the flat
        buffers (the bf16 copy of the biases it writes is unused)."""
        self.step_count += 1
        f = self.flat
        rsi.nn_adam(f["w"], f["m"], f["v"], f["g"], lr, self.step_count, self.flat16)

    def train_step(self, p, t, lr: float) -> torch.Tensor:
        self.forward(p)
        loss = self.loss(t)
        self.backward()
        self.adam(lr)
        return loss

    def predict(self, p) -> torch.Tensor:
        """Envelopes (scaled) for a batch of exactly B_alloc samples."""
        return self.forward(p)


# ---------------------------------------------------------------------------
# data from the RSI path, training, gate
# ---------------------------------------------------------------------------
def rsi_images(params, n_piston=1 << 14, n_iface=1 << 16, chunk=512, index0=0, device="cuda"):
    """Normalised images k phi / v0 (complex64 [n, 128, 128]) of the c5
    chains for each parameter row, computed by the batched RSI path."""
    out = []
    for c0 in range(0, len(params), chunk):
        cfgs = [W.c5_instance(params[i], index0 + i, n_piston, n_iface) for i in range(c0, min(len(params), c0 + chunk))]
        b = rsi.Batch(cfgs, seed=0, device=device)
        b.run()
        out.append(b.images.view(len(cfgs), 128, 128).clone())
        b.close()
        del b
    rsi.sync_status()
    return torch.cat(out, 0)


def _coeffs(params, device):
    """carrier_coeffs on the device: staged in pinned memory and copied
    without blocking, so the host does not wait for the kernels in flight."""
    host = torch.from_numpy(carrier_coeffs(params))
    if torch.device(device).type != "cuda":
        return host.to(device)
    return host.pin_memory().to(device, non_blocking=True)


def demodulate(images, params, device="cuda"):
    """Envelope = image * exp(-i psi), as interleaved f32 [n, 2*128*128]."""
    car = _coeffs(params, device)
    x = torch.view_as_real(images.contiguous()).reshape(images.shape[0], -1)
    out = torch.empty_like(x)
    rsi.nn_carrier(car, WINDOW, -1, x, out)
    return out


def modulate(env, params, device="cuda", scale: float = 1.0):
    """Image (complex64 [n, 128, 128]) from an interleaved envelope, times
    `scale` (the network's amplitude scale, applied in the same pass)."""
    car = _coeffs(params, device)
    out = torch.empty_like(env)
    rsi.nn_carrier(car, WINDOW, +1, env.contiguous(), out, scale=scale)
    return torch.view_as_complex(out.view(env.shape[0], 128, 128, 2))


def rel_errors(pred, ref):
    """Per-sample relative L2 error of complex images."""
    d = (pred - ref).reshape(pred.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    return (torch.linalg.vector_norm(d, dim=1) / torch.linalg.vector_norm(r, dim=1)).float()


class GraphedTrainer:
    """Training steps (forward, loss and its gradient, backward, Adam on every
    layer) of `net` replayed from one CUDA graph.  The graph reads the batch
    from fixed device buffers and Adam's (lr, 1 - beta1^t, 1 - beta2^t) from a
    device tensor (rsi_nn_adam_dev), which each step refreshes from a
    schedule held on the device, so nothing in a step waits for the host.
    The net must have taken one eager step (train_step) first: that step runs
    every kernel's one-time set-up, which a capture cannot hold."""

    BETA1, BETA2 = 0.9, 0.999

    def __init__(self, net: MLP, lrs):
        if net.step_count < 1:
            raise ValueError("GraphedTrainer needs one eager training step first")
        self.net = net
        dev, B = net.device, net.B_alloc
        self.p = torch.zeros(B, 5, dtype=torch.float32, device=dev)
        self.t = torch.zeros(B, net.y.shape[1], dtype=torch.float32, device=dev)
        self.hyper = torch.zeros(3, dtype=torch.float32, device=dev)
        # schedule row for step t (counted from the net's next step): lr and
        # the bias corrections, formed as rsi_nn_adam forms them (FP64 pow of
        # the FP32 betas, rounded to FP32)
        b1, b2 = float(np.float32(self.BETA1)), float(np.float32(self.BETA2))
        t0 = net.step_count + 1
        rows = [(lr, 1.0 - b1 ** (t0 + i), 1.0 - b2 ** (t0 + i)) for i, lr in enumerate(lrs)]
        self.sched = torch.tensor(np.asarray(rows, np.float32), device=dev)
        self.i = 0
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            net.forward(self.p)
            net.loss(self.t)
            net.backward()
            f = net.flat
            rsi.nn_adam_dev(f["w"], f["m"], f["v"], f["g"], self.hyper, net.flat16, self.BETA1, self.BETA2)

    def step(self, p_all, t_all, idx) -> torch.Tensor:
        """One step on rows idx (a device index tensor) of the training set;
        returns the device loss buffer."""
        if self.i >= len(self.sched):
            raise RuntimeError("GraphedTrainer: the learning-rate schedule is exhausted")
        torch.index_select(p_all, 0, idx, out=self.p)
        torch.index_select(t_all, 0, idx, out=self.t)
        self.hyper.copy_(self.sched[self.i])
        self.graph.replay()
        self.i += 1
        self.net.step_count += 1
        return self.net.loss_buf


class GraphedInference:
    """The surrogate's inference at a fixed batch (the network's B_alloc):
    carrier coefficients, Fourier features, hidden layers, output layer and
    the carrier pass with the amplitude scale, captured once into a CUDA
    graph and replayed per batch.  Each call stages the FP64 parameters in a
    pinned host buffer, copies them to a fixed device buffer without
    blocking, and replays the graph: one launch instead of eight calls
    through Python, so the batch runs at the kernels' speed.  With the
    tcgen05 engine the output layer applies the carrier in its epilogue
    (rsi_nn_gemm_carrier), so the layer's raw output never reaches memory.  The returned
    images (complex64 [B, 128, 128]) are a view of a buffer that the next
    call overwrites."""

    def __init__(self, net: MLP, scale: float):
        self.net, self.scale, self.B = net, float(scale), net.B_alloc
        dev = net.device
        self.p = torch.zeros(self.B, 5, dtype=torch.float32, device=dev)
        self.p64 = torch.zeros(self.B, 5, dtype=torch.float64, device=dev)
        self.car = torch.zeros(self.B, 4, dtype=torch.float64, device=dev)
        self.out = torch.empty(self.B, 2 * 128 * 128, dtype=torch.float32, device=dev)
        self.rows = torch.empty(8 * self.B, dtype=torch.float32, device=dev)  # carrier row constants
        self.p_host = torch.zeros(self.B, 5, dtype=torch.float64).pin_memory()
        self.copied = None  # event: the last call's host buffers have been read
        # one plain run first: the library's one-time set-up (kernel
        # attributes, the status word) happens outside the capture
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            self._body()
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body()

    def _body(self):
        net = self.net
        rsi.nn_carrier_coeffs(self.p64, C1, C2, self.car, self.p)
        if net.engine == "tcgen05":  # output layer and carrier in one kernel
            rsi.nn_gemm_carrier(net.hidden(self.p), net.W16[-1], net.b[-1], self.car, WINDOW, +1, self.scale,
                                self.out, workspace=self.rows)
        else:
            rsi.nn_carrier(self.car, WINDOW, +1, net.forward(self.p), self.out, scale=self.scale)

    def __call__(self, params) -> torch.Tensor:
        params = np.asarray(params, np.float64)
        if params.shape != (self.B, 5):
            raise ValueError(f"GraphedInference takes exactly {self.B} parameter rows")
        if self.copied is not None:
            self.copied.synchronize()  # the previous call's copies have read the host buffers
        self.p_host.numpy()[:] = params
        self.p64.copy_(self.p_host, non_blocking=True)
        self.copied = torch.cuda.Event()
        self.copied.record()
        self.graph.replay()
        return torch.view_as_complex(self.out.view(self.B, 128, 128, 2))


class Surrogate:
    """Trained network + held-out error table for the fallback gate."""

    def __init__(self, net: MLP, held_params, held_err, threshold=1e-2, k=8):
        self.net, self.threshold, self.k = net, threshold, k
        self.held_u = self._norm(held_params)
        self.held_err = np.asarray(held_err, np.float64)
        self._graph = None

    @staticmethod
    def _norm(params):
        return 2.0 * (np.asarray(params, np.float64) - LO) / (HI - LO) - 1.0

    def error_estimate(self, params) -> np.ndarray:
        """Mean held-out error of the k nearest held-out samples (in the
        normalised parameter box) of each query."""
        u = self._norm(params)
        d = ((u[:, None, :] - self.held_u[None, :, :]) ** 2).sum(-1)
        nn = np.argpartition(d, min(self.k, d.shape[1] - 1), axis=1)[:, :self.k]
        return self.held_err[nn].mean(axis=1)

    def infer(self, params, device="cuda"):
        """Images for params (batch = the network's batch): surrogate where
        the error estimate is within the threshold, RSI elsewhere.  The
        network runs through its CUDA graph (built on the first call)."""
        params = np.asarray(params, np.float64)
        if self._graph is None:
            self._graph = GraphedInference(self.net, self.net.scale)
        img = self._graph(params).clone()
        est = self.error_estimate(params)
        fall = np.nonzero(est > self.threshold)[0]
        if len(fall):
            img[torch.tensor(fall, device=device)] = rsi_images(params[fall], index0=10**6).to(img.dtype)
        return img, est, fall


def train(net: MLP, params, env, epochs: int, lr: float = 1e-3, seed: int = 0, log=None, graph: bool = True):
    """Adam on shuffled mini-batches of (params, scaled envelopes), cosine
    learning-rate decay.  With graph=True every step after the first is a
    replay of one CUDA graph (GraphedTrainer); the steps compute the same."""
    n = params.shape[0]
    B = net.B_alloc
    rng = np.random.default_rng(seed)
    p_all = torch.tensor(params, dtype=torch.float32, device=net.device)
    steps = (n // B) * epochs
    lrs = [lr * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps))) for s in range(steps)]
    total = 0
    trainer = None
    losses = []
    for ep in range(epochs):
        order = torch.tensor(rng.permutation(n)[: (n // B) * B], device=net.device).view(-1, B)
        for idx in order:
            if graph and total > 0:
                if trainer is None:
                    trainer = GraphedTrainer(net, lrs[total:])
                loss = trainer.step(p_all, env, idx)
            else:
                loss = net.train_step(p_all[idx], env[idx], lrs[total])
            total += 1
        losses.append(float(loss.item()))
        if log:
            log(ep, losses[-1])
    return losses
