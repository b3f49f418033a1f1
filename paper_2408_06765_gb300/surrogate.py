"""Learned surrogate of the RSI chain (not in the paper): a coordinate network
that gives the field image of one water -> steel chain for the inputs
(x-offset, tilt, water path L, frequency f, image depth d), trained on images
the GPU RSI path computes, with the RSI path as its fallback and the measure
of its error.

The network is evaluated per pixel (include/rsi.h, rsi_nn_net): each row
holds the field's parameters and the pixel's place in the window, recast in
the refracted beam's frame (Snell's law) and with the Fresnel number of the
equivalent water path; a Fourier-feature MLP (BF16 tensor-core GEMMs with FP32
accumulation) returns the pixel's carrier-demodulated field over the field's
RMS and the log of that RMS.  An image's pixels are not tied to a fixed
output basis, so a family of beams that turn through 0-90 degrees in the
steel, narrow with frequency and move with the window stays within reach: a
linear output layer of rank 512 over the 128 x 128 pixels leaves 12-19% of
held-out fields unexplained however it is trained.

Every numerical step runs in librsi.so (rsi_nn_rows, rsi_nn_forward,
rsi_nn_backward, rsi_nn_adam_step, rsi_nn_targets, rsi_nn_infer); this module
keeps the buffers, the training schedule and the fallback gate.  The FP64
oracle of the network is oracle/coordnet.py.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import rsi
from . import workloads as W

C1, C2 = W.WATER["c"], W.STEEL["c"]
A_PISTON = 6.35e-3
CRIT = math.asin(C1 / C2)  # critical angle of the water -> steel L wave
# box of (|tilt|, L, f, d) for the row inputs, and of the five inputs
BOX_LO = (0.0, 20e-3, 2e6, 1e-3)
BOX_HI = (math.radians(15.0), 60e-3, 10e6, 20e-3)
LO = np.array([-10e-3, math.radians(-15.0), 20e-3, 2e6, 1e-3])
HI = np.array([10e-3, math.radians(15.0), 60e-3, 10e6, 20e-3])
WINDOW = {"x0": -20e-3, "x1": 20e-3, "nx": 128, "z0": 0.0, "z1": 40e-3, "nz": 128}
NPIX = WINDOW["nx"] * WINDOW["nz"]


def fourier_matrix(n_freq: int, sigmas=(1.0, 4.0, 16.0), seed: int = 0) -> np.ndarray:
    """B [F][9]: Gaussian rows, split as evenly as possible over the scales."""
    rng = np.random.default_rng(seed)
    parts = np.array_split(np.arange(n_freq), len(sigmas))
    B = np.zeros((n_freq, rsi_in()), np.float32)
    for idx, sg in zip(parts, sigmas):
        B[idx] = rng.normal(0.0, sg, size=(len(idx), rsi_in()))
    return B


def rsi_in() -> int:
    return 9


class CoordNet:
    """Parameters (flat buffers: f32 weights, Adam moments, gradient, bf16
    copy), Fourier matrix and activation workspace of the coordinate network."""

    def __init__(self, n_freq=248, width=512, depth=5, rows=65536, sigmas=(1.0, 4.0, 16.0), seed=0,
                 engine="tcgen05", device="cuda"):
        self.device = device
        self.n_freq, self.width, self.depth, self.rows = n_freq, width, depth, rows
        self.fmat = torch.tensor(fourier_matrix(n_freq, sigmas, seed), device=device)
        self.net = rsi.nn_net_struct(n_freq, width, depth, rows, engine, C1, C2, A_PISTON, BOX_LO, BOX_HI,
                                     WINDOW, self.fmat)
        self.elems = rsi.nn_param_elems(self.net)
        f32 = dict(dtype=torch.float32, device=device)
        self.w = torch.zeros(self.elems, **f32)
        self.m = torch.zeros(self.elems, **f32)
        self.v = torch.zeros(self.elems, **f32)
        self.g = torch.zeros(self.elems, **f32)
        self.w16 = torch.zeros(self.elems, dtype=torch.bfloat16, device=device)
        rng = np.random.default_rng(seed + 1)
        for l in range(depth + 1):
            out, inp = self.shape(l)
            std = math.sqrt(2.0 / inp) if l < depth else math.sqrt(1.0 / inp)
            self.layer(l).copy_(torch.tensor(rng.normal(0.0, std, size=(out, inp)), **f32))
        rsi.nn_cast_bf16(self.w, self.w16)
        self.act = torch.empty(rsi.nn_act_bytes(self.net), dtype=torch.uint8, device=device)
        self.y = torch.zeros(rows, 4, **f32)
        self.loss = torch.zeros(1, **f32)
        self.hyper = torch.zeros(3, **f32)
        self.seed = torch.zeros(1, dtype=torch.int64, device=device)
        self.step_count = 0
        self._carrier = None

    def shape(self, l: int):
        inp = 2 * self.n_freq + 16 if l == 0 else self.width
        return (3 if l == self.depth else self.width), inp

    def layer(self, l: int, bias: bool = False, buf=None) -> torch.Tensor:
        """View of W_l ([out][in]) or b_l in a flat buffer (default: the weights)."""
        buf = self.w if buf is None else buf
        out, inp = self.shape(l)
        o = rsi.nn_param_offset(self.net, l, bias)
        return buf[o:o + out] if bias else buf[o:o + out * inp].view(out, inp)

    # -- one training step ----------------------------------------------------
    def rows_random(self, params64, targets, log_rms, seed: int | None = None):
        """Rows drawn at random over the training fields (seed: the device
        counter when None)."""
        rsi.nn_rows(self.net, params64, params64.shape[0], "random", self.act, seed=0 if seed is None else seed,
                    seed_dev=self.seed if seed is None else None, targets=targets, log_rms=log_rms)

    def forward(self):
        rsi.nn_forward(self.net, self.w16, self.w, self.act, self.y)
        return self.y

    def backward(self):
        rsi.nn_backward(self.net, self.w16, self.w, self.act, self.g, self.loss)
        return self.loss

    def adam(self):
        rsi.nn_adam_step(self.net, self.w, self.m, self.v, self.g, self.w16, self.hyper)

    # -- images ---------------------------------------------------------------
    def infer(self, params64, out=None) -> torch.Tensor:
        """Images (complex64 [n, nz, nx]) of the parameter rows (f64 [n, 5] on
        the device); the rows per call must hold whole fields."""
        n = params64.shape[0]
        if out is None:
            out = torch.empty(n, NPIX * 2, dtype=torch.float32, device=self.device)
        if self._carrier is None or self._carrier.shape[0] < n:
            self._carrier = torch.empty(n, 4, dtype=torch.float64, device=self.device)
        rsi.nn_infer(self.net, self.w16, self.w, params64, self.act, self._carrier, out)
        return torch.view_as_complex(out.view(n, WINDOW["nz"], WINDOW["nx"], 2))


class TrainingSet:
    """Training targets of RSI images on the device: each image demodulated by
    the refracted plane wave and divided by its RMS, and the log of the RMS
    (rsi_nn_targets)."""

    def __init__(self, net: CoordNet, params, images):
        dev = net.device
        self.params = torch.as_tensor(np.asarray(params, np.float64), device=dev)
        n = self.params.shape[0]
        self.targets = torch.empty(n, NPIX * 2, dtype=torch.float32, device=dev)
        self.log_rms = torch.empty(n, dtype=torch.float32, device=dev)
        carrier = torch.empty(n, 4, dtype=torch.float64, device=dev)
        p32 = torch.empty(n, 5, dtype=torch.float32, device=dev)
        env = torch.empty_like(self.targets)
        imgs = torch.view_as_real(images.contiguous()).reshape(n, -1)
        rsi.nn_targets(net.net, self.params, imgs, carrier, p32, env, self.targets, self.log_rms)


class GraphedTrainer:
    """Training steps (random rows, forward, backward, Adam) replayed from one
    CUDA graph.  Each step first copies its learning-rate row and row seed
    from schedules held on the device; nothing waits for the host.  The net
    must have taken one eager step first (kernel set-up outside the capture)."""

    BETA1, BETA2 = 0.9, 0.999

    def __init__(self, net: CoordNet, tset: TrainingSet, lrs, seeds):
        if net.step_count < 1:
            raise ValueError("GraphedTrainer needs one eager training step first")
        self.net, self.tset = net, tset
        dev = net.device
        b1, b2 = float(np.float32(self.BETA1)), float(np.float32(self.BETA2))
        t0 = net.step_count + 1
        rows = [(lr, 1.0 - b1 ** (t0 + i), 1.0 - b2 ** (t0 + i)) for i, lr in enumerate(lrs)]
        self.sched = torch.tensor(np.asarray(rows, np.float32), device=dev)
        self.seeds = torch.tensor(np.asarray(seeds, np.int64), device=dev)
        self.i = 0
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            net.rows_random(tset.params, tset.targets, tset.log_rms)
            net.forward()
            net.backward()
            net.adam()

    def step(self) -> torch.Tensor:
        if self.i >= len(self.sched):
            raise RuntimeError("GraphedTrainer: the learning-rate schedule is exhausted")
        self.net.hyper.copy_(self.sched[self.i])
        self.net.seed.copy_(self.seeds[self.i:self.i + 1])
        self.graph.replay()
        self.i += 1
        self.net.step_count += 1
        return self.net.loss


def train(net: CoordNet, tset: TrainingSet, steps: int, lr: float = 1e-3, warmup: int = 500, seed: int = 0,
          log=None, graph: bool = True):
    """Adam with a linear warm-up and cosine decay on random rows of the
    training set; with graph=True every step after the first replays one CUDA
    graph (GraphedTrainer).  Returns the losses every steps/20 steps."""
    lrs = [lr * min(1.0, (s + 1) / max(1, warmup)) * 0.5 * (1.0 + math.cos(math.pi * s / max(1, steps)))
           for s in range(steps)]
    b1, b2 = float(np.float32(GraphedTrainer.BETA1)), float(np.float32(GraphedTrainer.BETA2))
    seeds = np.random.default_rng(seed + 12345).integers(0, 2**62, size=steps, dtype=np.int64)
    losses = []
    # first step eagerly (one-time set-up of every kernel), then the graph
    net.hyper.copy_(torch.tensor([lrs[0], 1.0 - b1 ** (net.step_count + 1), 1.0 - b2 ** (net.step_count + 1)]))
    net.rows_random(tset.params, tset.targets, tset.log_rms, seed=int(seeds[0]))
    net.forward()
    net.backward()
    net.adam()
    net.step_count += 1
    trainer = GraphedTrainer(net, tset, lrs[1:], seeds[1:]) if graph and steps > 1 else None
    every = max(1, steps // 20)
    for s in range(1, steps):
        if trainer is not None:
            loss = trainer.step()
        else:
            b1t, b2t = 1.0 - b1 ** (net.step_count + 1), 1.0 - b2 ** (net.step_count + 1)
            net.hyper.copy_(torch.tensor([lrs[s], b1t, b2t]))
            net.rows_random(tset.params, tset.targets, tset.log_rms, seed=int(seeds[s]))
            net.forward()
            loss = net.backward()
            net.adam()
            net.step_count += 1
        if s % every == 0 or s == steps - 1:
            losses.append(float(loss.item()))
            if log:
                log(s, losses[-1])
    return losses


# ---------------------------------------------------------------------------
# the carrier: the refracted plane wave below the interface
# ---------------------------------------------------------------------------
def carrier_coeffs(params) -> np.ndarray:
    """(kx, kz, phi0, 0) per parameter row (numpy, FP64): psi = kx x + kz z +
    phi0 is the refracted plane wave's phase, x from the axis hit point and z
    below the window's top edge (the water path's phase k1 L included)."""
    p = np.atleast_2d(np.asarray(params, np.float64))
    k1 = 2 * np.pi * p[:, 3] / C1
    k2 = 2 * np.pi * p[:, 3] / C2
    s = C2 / C1 * np.sin(p[:, 1])
    c = np.sqrt(np.clip(1.0 - s * s, 0.0, None))
    return np.stack([k2 * s, k2 * c, k1 * p[:, 2] + k2 * c * p[:, 4], np.zeros(len(p))], axis=1)


def _coeffs(params, device):
    host = torch.from_numpy(carrier_coeffs(params))
    if torch.device(device).type != "cuda":
        return host.to(device)
    return host.pin_memory().to(device, non_blocking=True)


def demodulate(images, params, device="cuda"):
    """Images times exp(-i psi), as interleaved f32 [n, 2 nx nz] (rsi_nn_carrier)."""
    car = _coeffs(params, device)
    x = torch.view_as_real(images.contiguous()).reshape(images.shape[0], -1)
    out = torch.empty_like(x)
    rsi.nn_carrier(car, WINDOW, -1, x, out)
    return out


def modulate(env, params, device="cuda", scale: float = 1.0):
    """Images (complex64 [n, nz, nx]) from interleaved envelopes, times `scale`."""
    car = _coeffs(params, device)
    out = torch.empty_like(env)
    rsi.nn_carrier(car, WINDOW, +1, env.contiguous(), out, scale=scale)
    return torch.view_as_complex(out.view(env.shape[0], WINDOW["nz"], WINDOW["nx"], 2))


# ---------------------------------------------------------------------------
# data from the RSI path, errors, gate
# ---------------------------------------------------------------------------
def rsi_images(params, n_piston=1 << 16, n_iface=1 << 18, chunk=512, index0=0, device="cuda"):
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


def rel_errors(pred, ref):
    """Per-sample relative L2 error of complex images."""
    d = (pred - ref).reshape(pred.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    return (torch.linalg.vector_norm(d, dim=1) / torch.linalg.vector_norm(r, dim=1)).float()


class Surrogate:
    """Trained network + held-out error table for the fallback gate."""

    def __init__(self, net: CoordNet, held_params, held_err, threshold=1e-2, k=8, tilt_max=None):
        """tilt_max (radians): the largest |tilt| the network was trained on;
        queries beyond it always go to the RSI path (the network extrapolates
        there, its log-RMS output without bound)."""
        self.net, self.threshold, self.k, self.tilt_max = net, threshold, k, tilt_max
        self.held_u = self._norm(held_params)
        self.held_err = np.asarray(held_err, np.float64)

    @staticmethod
    def _norm(params):
        return 2.0 * (np.asarray(params, np.float64) - LO) / (HI - LO) - 1.0

    def error_estimate(self, params) -> np.ndarray:
        """Mean held-out error of the k nearest held-out samples (in the
        normalised parameter box, x-offset left out: the field does not depend
        on it) of each query."""
        u = self._norm(params)[:, 1:]
        h = self.held_u[:, 1:]
        d = ((u[:, None, :] - h[None, :, :]) ** 2).sum(-1)
        nn = np.argpartition(d, min(self.k, d.shape[1] - 1), axis=1)[:, :self.k]
        est = self.held_err[nn].mean(axis=1)
        if self.tilt_max is not None:
            est[np.abs(np.asarray(params, np.float64)[:, 1]) >= self.tilt_max] = np.inf
        return est

    def infer(self, params, device="cuda"):
        """Images for params: the network where the error estimate is within
        the threshold, the RSI path elsewhere.  Returns (images, estimates,
        indices of the queries sent to the RSI path)."""
        params = np.asarray(params, np.float64)
        img = self.net.infer(torch.tensor(params, device=device)).clone()
        est = self.error_estimate(params)
        fall = np.nonzero(est > self.threshold)[0]
        if len(fall):
            img[torch.tensor(fall, device=device)] = rsi_images(params[fall], index0=10**6).to(img.dtype)
        return img, est, fall
