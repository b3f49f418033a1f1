"""Several frequencies per stage on shared points (rsi_propagate_stage_multi)
against the single-frequency stages and the FP64 oracle: both stage kinds,
flat and per-point normals, launch shapes, a chain, and the full-size c2
frequencies against their stored oracle pixels."""
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
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def host(p):
    torch.cuda.synchronize()
    return {k: p.field(k.upper()).cpu().numpy() for k in ("x", "y", "z", "nx", "ny", "nz", "w")}


@pytest.mark.parametrize("nf", [2, 3, 4])
@pytest.mark.parametrize("case", ["piston", "rsi_flat", "rsi_curved"])
@pytest.mark.parametrize("shape", [{}, {"tile": 32, "splits": 3}, {"tile": 128, "splits": 1, "variant": 2}])
def test_multi_matches_single_stages_and_oracle(nf, case, shape):
    freqs = [1.7e6, 3.1e6, 5.5e6, 9.2e6][:nf]
    if case == "piston":
        src = rsi.make_qmc_points({"kind": "disk", "centre": (0.0, 0.0, 0.0), "tilt": 0.12, "a": 5e-3}, 0, 0, 3001)
        tgt = rsi.make_qmc_points({"kind": "rect", "centre": (0.0, 0.0, 0.03), "wx": 0.03, "wy": 0.03}, 0, 1, 1999)
        c, sig, kind, normals = 1480.0, None, rsi.STAGE_PISTON, rsi.NORMALS_Z
    else:
        curved = case == "rsi_curved"
        surf = {"kind": "cyl", "centre": (0.0, 0.0, 0.02), "wx": 0.03, "wy": 0.03, "R": 0.05} if curved else \
            {"kind": "rect", "centre": (0.0, 0.0, 0.02), "wx": 0.03, "wy": 0.03}
        src = rsi.make_qmc_points(surf, 0, 2, 4099)
        tgt = rsi.grid_points({"x0": -0.01, "x1": 0.012, "nx": 41, "z0": 0.021, "z1": 0.04, "nz": 33, "y": 0.0})
        rng = np.random.default_rng(nf)
        sig = torch.tensor(rng.normal(size=(nf, src.n)) + 1j * rng.normal(size=(nf, src.n)),
                           dtype=torch.complex128, device="cuda")
        c, kind = 5900.0, rsi.STAGE_RSI
        normals = rsi.NORMALS_POINTS if curved else rsi.NORMALS_Z
    ks = [2 * math.pi * f / c for f in freqs]
    st = rsi.stage_struct(kind, "fp32c", ks[0], 1.0, normals, **shape)
    got = rsi.propagate_stage_multi(st, ks, src, sig, tgt).cpu().numpy()
    rsi.sync_status()
    hs = host(src)
    tq = {k: v for k, v in host(tgt).items() if k in ("x", "y", "z")}
    packed = shape.get("variant", 0) != 2
    for f, k in enumerate(ks):
        one = rsi.stage_struct(kind, "fp32c", k, 1.0, normals, **dict(shape, variant=3 if packed else 2))
        single = rsi.propagate_stage(one, src, None if sig is None else sig[f].contiguous(), tgt).cpu().numpy()
        # the same arithmetic per frequency (the packed form sums in a different order)
        assert rel(got[f], single) < (2e-5 if packed else 1e-6), f
        want = oracle.piston_field(hs, tq, k) if sig is None else oracle.rsi_field(hs, sig[f].cpu().numpy(), tq, k)
        assert_close(got[f], want, 1e-4, f"frequency {f}")


@pytest.mark.parametrize("case", ["piston", "rsi_flat", "rsi_curved"])
@pytest.mark.parametrize("shape", [{}, {"tile": 32, "splits": 3}])
def test_shared_harmonic_matches_single_stages_and_oracle(case, shape):
    """Three frequencies of which one is twice another (6.2 = 2 x 3.1 MHz,
    given first, its base last, so the kernel reorders them): the far path
    forms the 6.2 MHz term from the 3.1 MHz one by the double angle, and every
    frequency still equals its single-frequency stage and the oracle."""
    freqs = [6.2e6, 1.7e6, 3.1e6]
    if case == "piston":
        src = rsi.make_qmc_points({"kind": "disk", "centre": (0.0, 0.0, 0.0), "tilt": 0.12, "a": 5e-3}, 0, 0, 3001)
        tgt = rsi.make_qmc_points({"kind": "rect", "centre": (0.0, 0.0, 0.03), "wx": 0.03, "wy": 0.03}, 0, 1, 1999)
        c, sig, kind, normals = 1480.0, None, rsi.STAGE_PISTON, rsi.NORMALS_Z
    else:
        curved = case == "rsi_curved"
        surf = {"kind": "cyl", "centre": (0.0, 0.0, 0.02), "wx": 0.03, "wy": 0.03, "R": 0.05} if curved else \
            {"kind": "rect", "centre": (0.0, 0.0, 0.02), "wx": 0.03, "wy": 0.03}
        src = rsi.make_qmc_points(surf, 0, 2, 4099)
        tgt = rsi.grid_points({"x0": -0.01, "x1": 0.012, "nx": 41, "z0": 0.021, "z1": 0.04, "nz": 33, "y": 0.0})
        rng = np.random.default_rng(7)
        sig = torch.tensor(rng.normal(size=(3, src.n)) + 1j * rng.normal(size=(3, src.n)),
                           dtype=torch.complex128, device="cuda")
        c, kind = 5900.0, rsi.STAGE_RSI
        normals = rsi.NORMALS_POINTS if curved else rsi.NORMALS_Z
    ks = [2 * math.pi * f / c for f in freqs]
    st = rsi.stage_struct(kind, "fp32c", ks[0], 1.0, normals, **shape)
    assert rsi.stage_multi_shared_harmonic(st, ks)
    assert not rsi.stage_multi_shared_harmonic(st, [ks[0] * (1 + 1e-9)] + ks[1:])
    assert not rsi.stage_multi_shared_harmonic(rsi.stage_struct(kind, "fp32c", ks[0], 1.0, normals, variant=2), ks)
    got = rsi.propagate_stage_multi(st, ks, src, sig, tgt).cpu().numpy()
    rsi.sync_status()
    hs = host(src)
    tq = {k: v for k, v in host(tgt).items() if k in ("x", "y", "z")}
    for f, k in enumerate(ks):
        one = rsi.stage_struct(kind, "fp32c", k, 1.0, normals, **dict(shape, variant=3))
        single = rsi.propagate_stage(one, src, None if sig is None else sig[f].contiguous(), tgt).cpu().numpy()
        assert rel(got[f], single) < 2e-5, f
        want = oracle.piston_field(hs, tq, k) if sig is None else oracle.rsi_field(hs, sig[f].cpu().numpy(), tq, k)
        assert_close(got[f], want, 1e-4, f"frequency {f}")


def test_reversed_normals_and_rejections():
    src = rsi.make_qmc_points({"kind": "rect", "centre": (0.0, 0.0, 0.02), "wx": 0.02, "wy": 0.02}, 0, 3, 2000)
    tgt = rsi.grid_points({"x0": -0.01, "x1": 0.01, "nx": 16, "z0": 0.0, "z1": 0.015, "nz": 16, "y": 0.0})
    sig = torch.ones((2, src.n), dtype=torch.complex128, device="cuda")
    ks = [2 * math.pi * 2e6 / 1480.0, 2 * math.pi * 3e6 / 1480.0]
    a = rsi.propagate_stage_multi(rsi.stage_struct(rsi.STAGE_RSI, "fp32c", ks[0], 1.0, rsi.NORMALS_Z), ks, src, sig,
                                  tgt)
    b = rsi.propagate_stage_multi(rsi.stage_struct(rsi.STAGE_RSI, "fp32c", ks[0], 1.0, rsi.NORMALS_NEG_Z), ks, src,
                                  sig, tgt)
    torch.cuda.synchronize()
    assert torch.equal(b, -a)
    with pytest.raises(rsi.RSIError):
        rsi.propagate_stage_multi(rsi.stage_struct(rsi.STAGE_RSI, "fp32c", ks[0]), ks * 3, src,
                                  torch.ones((6, src.n), dtype=torch.complex128, device="cuda"), tgt)
    with pytest.raises(rsi.RSIError):
        rsi.propagate_stage_multi(rsi.stage_struct(rsi.STAGE_RSI, "fp64", ks[0]), ks, src, sig, tgt)
    cfgs = [W.small_ragged("fp32c", freq=f) for f in (2e6, 3e6)]
    cfgs[1]["piston"] = dict(cfgs[1]["piston"], n=cfgs[1]["piston"]["n"] + 1)
    with pytest.raises(ValueError):
        rsi.run_chain_multi(cfgs)


def test_chain_multi_matches_oracle():
    cfgs = [W.small_ragged("fp32c", freq=f) for f in (2.5e6, 4e6, 7.5e6)]
    imgs = rsi.run_chain_multi(cfgs)
    torch.cuda.synchronize()
    rsi.sync_status()
    for cfg, img in zip(cfgs, imgs):
        want, _ = oracle.chain(cfg)
        k_last = oracle.wavenumber(cfg["freq"], cfg["media"][-1]["c"])
        assert_close(img.cpu().numpy(), k_last * want, 1e-4)
        single = rsi.run_chain(cfg).image
        assert rel(img.cpu().numpy(), single.cpu().numpy()) < 2e-5


def test_c2_frequencies_together_match_stored_oracle():
    cfgs = W.c2_all()
    imgs = rsi.run_chain_multi(cfgs)
    torch.cuda.synchronize()
    rsi.sync_status()
    for cfg, img in zip(cfgs, imgs):
        path = os.path.join(HERE, f"c2_{cfg['freq'] / 1e6:g}MHz.json")
        if not os.path.exists(path):
            pytest.skip("no stored oracle values")
        rec = json.load(open(path))
        got = img.reshape(-1).cpu().numpy()[np.asarray(rec["pixels"])]
        want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
        assert_close(got, want, 1e-4, path)
