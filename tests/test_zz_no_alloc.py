"""rsi_propagate_stage_noalloc, the stage entry point for callers that cannot
provide device scratch memory (see include/rsi.h), against the ordinary
workspace entry point rsi_propagate_stage.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes
import math

import numpy as np
import pytest
import torch

from paper_2408_06765_gb300 import build, rsi

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-5, "fp32c": 1e-4}
RSI_E_NOMEM = -5


@pytest.fixture(scope="module")
def noalloc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load().rsi_propagate_stage_noalloc  # argument types set by the binding


def rel_l2(a, b):
    a, b = a.cpu().numpy().ravel(), b.cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_noalloc_matches_workspace_entry(noalloc, prec):
    pist = rsi.make_qmc_points({"kind": "disk", "centre": (0.0, 0.0, 0.0), "a": 6.35e-3}, 0, 0, 3000)
    iface = rsi.make_qmc_points({"kind": "rect", "centre": (0.0, 0.0, 0.03), "wx": 0.05, "wy": 0.05},
                                0, 1, 20000)
    grid = rsi.grid_points({"x0": -0.02, "x1": 0.02, "nx": 96, "z0": 0.03, "z1": 0.07, "nz": 80})
    k1, k2 = 2 * math.pi * 5e6 / 1480.0, 2 * math.pi * 5e6 / 5900.0
    st1 = rsi.stage_struct(rsi.STAGE_PISTON, prec, k1)
    st2 = rsi.stage_struct(rsi.STAGE_RSI, prec, k2, normals=rsi.NORMALS_Z)
    ref1 = rsi.propagate_stage(st1, pist, None, iface)
    sigma = ref1.clone()
    ref2 = rsi.propagate_stage(st2, iface, sigma, grid)
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row reuse the static scratch
        out1 = torch.full_like(ref1, float("nan"))
        out2 = torch.full_like(ref2, float("nan"))
        rc = noalloc(ctypes.byref(st1), pist.ptr(), pist.n, None, iface.ptr(), iface.n,
                     ctypes.c_void_p(out1.data_ptr()), stream())
        assert rc == 0, rsi.load().rsi_last_error()
        rc = noalloc(ctypes.byref(st2), iface.ptr(), iface.n, ctypes.c_void_p(sigma.data_ptr()),
                     grid.ptr(), grid.n, ctypes.c_void_p(out2.data_ptr()), stream())
        assert rc == 0, rsi.load().rsi_last_error()
        torch.cuda.synchronize()
        rsi.sync_status()
        assert rel_l2(out1, ref1) <= TOL[prec]
        assert rel_l2(out2, ref2) <= TOL[prec]


def test_noalloc_rejects_stages_beyond_the_static_area(noalloc):
    # 2^22 FP64 sources need ~270 MB of staged tiles: rejected before any launch
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = rsi.stage_struct(rsi.STAGE_RSI, "fp64", 1000.0, normals=rsi.NORMALS_Z)
    rc = noalloc(ctypes.byref(st), p, 1 << 22, p, p, 1 << 10, p, stream())
    assert rc == RSI_E_NOMEM
    assert b"static area" in rsi.load().rsi_last_error()


def test_noalloc_lowers_the_split_count_to_fit(noalloc):
    """With splits = 0, a stage whose automatic split count would need more
    partial-sum space than the static area holds runs with fewer splits: the
    same field as the workspace entry point.  1.9 million piston sources in
    32-source tiles (32-byte header + 32 records of 32 bytes) take 59.8 MiB
    of the 64 MiB area, so at most eight splits of 2^15 targets (0.5 MiB of
    partial sums each) fit beside them, while the automatic count for 64
    target blocks asks for more."""
    L = rsi.load()
    n_src = 1_900_000
    pist = rsi.make_qmc_points({"kind": "disk", "centre": (0.0, 0.0, 0.0), "a": 6.35e-3}, 0, 0, n_src)
    grid = rsi.grid_points({"x0": -0.02, "x1": 0.02, "nx": 256, "z0": 0.03, "z1": 0.07, "nz": 128})
    k1 = 2 * math.pi * 5e6 / 1480.0
    st = rsi.stage_struct(rsi.STAGE_PISTON, "fp32c", k1, tile=32)
    auto = L.rsi_stage_workspace_bytes(ctypes.byref(st), pist.n, grid.n)
    one = rsi.stage_struct(rsi.STAGE_PISTON, "fp32c", k1, tile=32, splits=1)
    tiles_only = L.rsi_stage_workspace_bytes(ctypes.byref(one), pist.n, grid.n)
    area = 64 << 20
    assert auto > area >= tiles_only, (auto, tiles_only)  # the case this test is about
    ref = rsi.propagate_stage(st, pist, None, grid)
    torch.cuda.synchronize()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        rc = noalloc(ctypes.byref(st), pist.ptr(), pist.n, None, grid.ptr(), grid.n,
                     ctypes.c_void_p(out.data_ptr()), stream())
        assert rc == 0, L.rsi_last_error()
        torch.cuda.synchronize()
        rsi.sync_status()
        assert rel_l2(out, ref) <= TOL["fp32c"]
