"""f3/f4 sources on the GPU against the FP64 oracle: Halton point sets
(bit-exact integer coordinates, index order), the focused transducer's
spherical cap and the Gaussian apodisation (FP64 geometry within a few
ulps), and whole chains with them: Halton sets and an apodised piston
through the c1 geometry, the focused transducer through the RSI chain and
the ray-tracing model."""
import ctypes
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


def host(p):
    torch.cuda.synchronize()
    out = {k: p.field(k).cpu().numpy() for k in ("X", "Y", "Z", "NX", "NY", "NZ", "W")}
    for k in ("IDX", "SU", "SV"):
        out[k] = p.field(k).cpu().numpy().view(np.uint32)
    return out


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


SURFS = [
    {"kind": "disk", "centre": (1e-3, -2e-3, 0.5e-3), "tilt": math.radians(11.0), "a": 6.35e-3},
    {"kind": "rect", "centre": (2e-3, 0.0, 0.05), "wx": 0.06, "wy": 0.04},
    {"kind": "cyl", "centre": (0.0, 0.0, 0.03), "wx": 0.06, "wy": 0.06, "R": 0.1},
    {"kind": "cap", "centre": (1e-3, 0.0, 0.0), "tilt": math.radians(7.0), "a": 6.35e-3, "R": 33e-3},
    {"kind": "cap", "centre": (0.0, 1e-3, 0.0), "tilt": 0.0, "a": 6.35e-3, "R": 33e-3, "apod": 4e-3},
    {"kind": "disk", "centre": (0.0, 0.0, 0.0), "tilt": 0.0, "a": 6.35e-3, "apod": 3e-3},
]


def check_geometry(p, ref, order, surf):
    extent = sum(abs(c) for c in surf["centre"]) + 2 * max(surf.get(k, 0.0) for k in ("a", "wx", "wy", "R"))
    for key in ("x", "y", "z", "nx", "ny", "nz", "w"):
        got, want = p[key.upper()], ref[key][order]
        scale = extent if key in ("x", "y", "z") else float(np.max(np.abs(want)))
        assert np.max(np.abs(got - want)) <= 8 * 2.0 ** -52 * scale + 1e-300, key


@pytest.mark.parametrize("surf", SURFS, ids=lambda s: s["kind"] + ("_apod" if s.get("apod") else ""))
@pytest.mark.parametrize("n", [1, 7, 1000, 3 ** 7 + 5])
def test_halton_points(surf, n):
    s = dict(surf, sequence="halton")
    p = host(rsi.make_qmc_points(s, 0, 0, n))
    assert np.array_equal(p["IDX"], np.arange(1, n + 1, dtype=np.uint32))  # index order, points 1..n
    su, sv = oracle.halton(n)
    assert np.array_equal(p["SU"], su) and np.array_equal(p["SV"], sv)
    check_geometry(p, oracle.map_points(s, su, sv), np.arange(n), s)


@pytest.mark.parametrize("surf", SURFS[3:], ids=["cap_tilted", "cap_apod", "disk_apod"])
@pytest.mark.parametrize("n,seed,set_id", [(5, 0, 1), (4096, 2, 3), (65536 + 77, 0, 4)])
def test_sobol_cap_and_apodised_points(surf, n, seed, set_id):
    p = host(rsi.make_qmc_points(surf, seed, set_id, n))
    idx = p["IDX"]
    su, sv = oracle.sobol(seed, set_id, n)
    assert np.array_equal(p["SU"], su[idx]) and np.array_equal(p["SV"], sv[idx])
    check_geometry(p, oracle.map_points(surf, su, sv), idx, surf)


def test_halton_rejects_scrambling():
    s = rsi.surface_struct(dict(SURFS[0], sequence="halton"))
    s.scramble = 1
    pts = rsi.Points(16)
    rc = rsi.load().rsi_make_qmc_points(ctypes.byref(s), 0, 0, 16, pts.ptr(), pts.nbytes, None)
    assert rc != 0


@pytest.mark.parametrize("apod", [0.0, 4e-3])
def test_halton_chain_matches_oracle(apod):
    cfg = W.f3_halton(apod)
    img = rsi.run_chain(cfg).image
    torch.cuda.synchronize()
    rsi.sync_status()
    want, _ = oracle.chain(cfg)
    k2 = oracle.wavenumber(cfg["freq"], cfg["media"][1]["c"])
    assert_close(img.cpu().numpy(), k2 * want, 1e-4)


def test_focused_chain_and_ray_tracing_match_oracle():
    cfg = W.f4_small()
    img = rsi.run_chain(cfg).image.cpu().numpy()
    want, _ = oracle.chain(cfg)
    k2 = oracle.wavenumber(cfg["freq"], cfg["media"][1]["c"])
    assert_close(img, k2 * want, 1e-4)
    ray = rsi.run_raytrace(cfg).cpu().numpy()
    assert_close(ray, oracle.raytrace_image(cfg), 1e-4)
    rsi.sync_status()


@pytest.mark.parametrize("name", ["f4_chain_2.5MHz", "f4_ray_2.5MHz"])
def test_focused_full_size_matches_stored_oracle(name):
    path = os.path.join(HERE, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle values for {name}")
    rec = json.load(open(path))
    cfg = W.f4_focused()
    img = rsi.run_chain(cfg).image if "chain" in name else rsi.run_raytrace(cfg)
    torch.cuda.synchronize()
    rsi.sync_status()
    got = img.reshape(-1).cpu().numpy()[np.asarray(rec["pixels"])]
    want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
    assert_close(got, want, 1e-4, name)
