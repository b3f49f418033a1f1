"""The ray-tracing model (Sec. 2.2, Eq. transmitted_ray_tracing) on the GPU
against the FP64 oracle: a small ragged case reaching steep refraction
angles, launch shapes, one medium against the GPU piston stage, and stored
oracle pixels of the full-size f2 workload in the launch shape bench.py
times."""
import json
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
TOL = 1e-4  # FP32 pair arithmetic with a double-float reference phase per (target, tile)


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load()


def rel(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_small_case_matches_oracle():
    cfg = W.f2_small()
    img = rsi.run_raytrace(cfg)
    torch.cuda.synchronize()
    rsi.sync_status()
    want = oracle.raytrace_image(cfg)
    err = rel(img.cpu().numpy(), want)
    assert err < TOL, err
    # every pixel, not only the norm: the worst one within 1e-3 of the image's largest value
    assert np.max(np.abs(img.cpu().numpy() - want)) < 1e-3 * np.max(np.abs(want))


@pytest.mark.parametrize("tile,splits,newton", [(32, 1, 0), (64, 3, 0), (256, 7, 0), (0, 0, 6)])
def test_launch_shapes_agree(tile, splits, newton):
    cfg = W.f2_small()
    ref = rsi.run_raytrace(cfg).cpu().numpy()
    got = rsi.run_raytrace(cfg, tile=tile, splits=splits, newton=newton).cpu().numpy()
    torch.cuda.synchronize()
    assert rel(got, ref) < 2e-5
    assert_close(got, oracle.raytrace_image(cfg), TOL)


def test_one_medium_equals_the_piston_stage():
    # identical media: straight rays, T12 = 1 and the spreading is r, so the
    # model is Eq. incident_field itself
    cfg = W.f2_small()
    cfg["media"] = [dict(W.WATER), dict(W.WATER)]
    img = rsi.run_raytrace(cfg)
    seed, pc = 0, cfg["piston"]
    pts = rsi.make_qmc_points(dict(pc, kind="disk"), seed, 0, int(pc["n"]))
    tgt = rsi.grid_points(cfg["grid"])
    k = rsi.wavenumber(cfg["freq"], W.WATER["c"])
    phi = rsi.propagate_stage(rsi.stage_struct(rsi.STAGE_PISTON, "fp64", k, 1.0), pts, None, tgt)
    direct = rsi.field_image(cfg["grid"], phi, k)
    torch.cuda.synchronize()
    assert rel(img.cpu().numpy(), direct.cpu().numpy()) < TOL


def test_full_size_matches_stored_oracle():
    path = os.path.join(HERE, "f2_5MHz.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle values for f2_5MHz")
    rec = json.load(open(path))
    img = rsi.run_raytrace(W.f2_ray_tracing())
    torch.cuda.synchronize()
    rsi.sync_status()
    got = img.reshape(-1).cpu().numpy()[np.asarray(rec["pixels"])]
    want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
    assert_close(got, want, TOL)
