"""The target-sharded chain on the GPU: every rank of a sharded chain run in
one process, one after another (shard.run_emulated: the all-gathers become
concatenations, so no rank waits for another), with the stage sums in
librsi's kernels on slices cut by rsi_points_slice.  The assembled images
equal the one-rank chain's (FP64: to rounding; FP32C: within the split
regrouping of the sums) and the FP64 oracle's."""
import numpy as np
import pytest
import torch

import oracle
from fieldcheck import assert_close
from paper_2408_06765_gb300 import build, rsi, shard
from paper_2408_06765_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load()


def test_points_slice_copies_every_field():
    pts = rsi.make_qmc_points({"kind": "cyl", "centre": (0.0, 0.0, 0.03), "wx": 0.03, "wy": 0.02, "R": 0.05},
                              0, 3, 1001)
    sub = rsi.points_slice(pts, 217, 333)
    torch.cuda.synchronize()
    for name in rsi.PF:
        assert torch.equal(sub.field(name), pts.field(name)[217:217 + 333]), name
    with pytest.raises(rsi.RSIError):
        rsi.points_slice(pts, 900, 200)


@pytest.mark.parametrize("world", [1, 2, 5])
def test_sharded_fp64_chain_equals_one_rank(world):
    cfg = W.c3_multilayer(curved=True, n_per_surface=700)
    cfg["precision"] = "fp64"
    cfg["grid"] = dict(cfg["grid"], nx=31, nz=19)
    be = shard.LibrsiBackend("fp64")
    img = shard.assemble(shard.run_emulated([cfg], world, be), be)[0]
    one = rsi.run_chain(cfg).image
    torch.cuda.synchronize()
    rsi.sync_status()
    assert_close(img.cpu().numpy(), one.cpu().numpy(), 1e-12)
    assert_close(img.cpu().numpy(), oracle.field_image(cfg), 1e-5)


def test_sharded_frequencies_equal_the_multi_frequency_chain():
    cfgs = [W.small_ragged("fp32c", freq=f) for f in (2.5e6, 4e6, 7.5e6)]
    be = shard.LibrsiBackend("fp32c")
    imgs = shard.assemble(shard.run_emulated(cfgs, 3, be), be)
    one = rsi.run_chain_multi(cfgs)
    torch.cuda.synchronize()
    rsi.sync_status()
    for f, cfg in enumerate(cfgs):
        assert_close(imgs[f].cpu().numpy(), one[f].cpu().numpy(), 1e-5)
        assert_close(imgs[f].cpu().numpy(), oracle.field_image(cfg), 1e-4)
