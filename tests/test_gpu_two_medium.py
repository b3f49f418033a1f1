"""Reflected field in medium 1 and the two-medium image on the GPU (the
reflected field on the interface taken as R12 times the incident field,
Sec. 2.1), against the FP64 oracle: the source density R12 phi, the stage
with reversed normals, the whole image on a small ragged case, and stored
oracle pixels of the full-size f1 workload in the launch shapes bench.py
times."""
import json
import math
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2408_06765_gb300 import build, rsi
from paper_2408_06765_gb300 import workloads as W
from fieldcheck import assert_close

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def host_points(p: rsi.Points) -> dict:
    return {k: p.field(k.upper()).cpu().numpy() for k in ("x", "y", "z", "nx", "ny", "nz", "w")}


@pytest.mark.parametrize("mode,tilt_deg", [("global", 0.0), ("global", 10.0), ("global", 20.0),
                                           ("local", 8.0)])
def test_reflect_matches_oracle(mode, tilt_deg):
    surf = {"kind": "cyl", "centre": (1e-3, 0.0, 30e-3), "wx": 40e-3, "wy": 40e-3, "R": 60e-3} \
        if mode == "local" else {"kind": "rect", "centre": (0.0, 0.0, 30e-3), "wx": 40e-3, "wy": 40e-3}
    n = 1237
    pts = rsi.make_qmc_points(surf, 0, 3, n)
    rng = np.random.default_rng(7)
    phi = rng.normal(size=n) + 1j * rng.normal(size=n)
    phi_d = torch.tensor(phi, dtype=torch.complex128, device="cuda")
    C = math.sin(math.radians(tilt_deg)) / W.WATER["c"]
    got = rsi.interface_reflect(pts, phi_d, W.WATER, W.STEEL, C, mode).cpu().numpy()
    torch.cuda.synchronize()
    want, _ = oracle.reflect(host_points(pts), phi, W.WATER, W.STEEL, C, mode)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("precision", ["fp64", "fp32c"])
@pytest.mark.parametrize("surf", ["rect", "cyl"])
def test_reversed_normals_negate_the_stage(precision, surf):
    s = {"kind": "cyl", "centre": (0.0, 0.0, 20e-3), "wx": 30e-3, "wy": 30e-3, "R": 50e-3} if surf == "cyl" \
        else {"kind": "rect", "centre": (0.0, 0.0, 20e-3), "wx": 30e-3, "wy": 30e-3}
    src = rsi.make_qmc_points(s, 0, 1, 3001)
    tgt = rsi.grid_points({"x0": -10e-3, "x1": 10e-3, "nx": 37, "z0": 2e-3, "z1": 15e-3, "nz": 29, "y": 0.0})
    rng = np.random.default_rng(3)
    sig = torch.tensor(rng.normal(size=3001) + 1j * rng.normal(size=3001), dtype=torch.complex128, device="cuda")
    k = 2 * math.pi * 5e6 / 1480.0
    pos, neg = (rsi.NORMALS_Z, rsi.NORMALS_NEG_Z) if surf == "rect" else (rsi.NORMALS_POINTS, rsi.NORMALS_POINTS_NEG)
    a = rsi.propagate_stage(rsi.stage_struct(rsi.STAGE_RSI, precision, k, 1.0, pos), src, sig, tgt)
    b = rsi.propagate_stage(rsi.stage_struct(rsi.STAGE_RSI, precision, k, 1.0, neg), src, sig, tgt)
    torch.cuda.synchronize()
    assert torch.equal(b, -a)  # IEEE negation commutes with every product and sum
    want = oracle.rsi_field(oracle.flip_normals(host_points(src)), sig.cpu().numpy(),
                            {key: tgt.field(key.upper()).cpu().numpy() for key in ("x", "y", "z")}, k)
    assert rel(b.cpu().numpy(), want) < (1e-12 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32c", 1e-4)])
def test_two_medium_small_matches_oracle(precision, tol):
    cfg = W.f1_small()
    res = rsi.run_two_medium(cfg, precision=precision)
    torch.cuda.synchronize()
    rsi.sync_status()
    want = oracle.two_medium(cfg)
    got = res.image.cpu().numpy()
    assert got.shape == want.shape
    nw = cfg["grid_water"]["nz"]
    assert_close(got[:nw], want[:nw], tol, "water window (incident + reflected)")
    assert_close(got[nw:], want[nw:], tol, "steel window (transmitted)")
    parts = oracle.two_medium(cfg, parts=True)
    assert_close(res.parts["reflected"].cpu().numpy(), parts["reflected"], tol, "reflected")


def test_two_medium_full_size_matches_stored_oracle():
    path = os.path.join(HERE, "f1_5MHz.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle values for f1_5MHz")
    rec = json.load(open(path))
    res = rsi.run_two_medium(W.f1_two_medium())
    torch.cuda.synchronize()
    rsi.sync_status()
    got = res.image.reshape(-1).cpu().numpy()[np.asarray(rec["pixels"])]
    want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
    assert_close(got, want, 1e-4)
