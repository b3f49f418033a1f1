"""Host-side planning of batched chains (no GPU needed): rsi_batch_create
lays out the workspace and rejects invalid instances before any launch."""
import copy

import pytest

from paper_2408_06765_gb300 import build, rsi
from paper_2408_06765_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return rsi.load()


def test_c4_plan_layout():
    cfgs = W.c4_all()
    assert len(cfgs) == 2048
    b = rsi.Batch(cfgs, allocate=False)
    try:
        assert b.image_elems == 2048 * 128 * 128
        # points + fields + tiles + partial sums of 2048 uneven instances fit easily in HBM
        assert 1e9 < b.workspace_bytes < 40e9
        assert b.offsets[1] == 128 * 128
    finally:
        b.close()


def test_c4_counts_are_log_uniform_and_seeded():
    c = W.c4_counts()
    assert c.shape == (2048, 2) and c.min() >= 4096 and c.max() <= 65536
    assert (W.c4_counts() == c).all()
    import numpy as np
    u = (np.log2(c) - 12.0) / 4.0
    assert abs(u.mean() - 0.5) < 0.03


@pytest.mark.parametrize("bad", ["piston_rect", "no_points", "two_interfaces", "fp64"])
def test_plan_rejects_invalid(bad):
    cfg = W.small_ragged("fp32c")
    shape = None
    if bad == "piston_rect":
        inst = rsi.batch_instance(cfg)
        inst.piston.kind = rsi.SURF["rect"]
        arr = (rsi.BatchInstance * 1)(inst)
        import ctypes
        plan, ws, n = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_size_t()
        rc = rsi.load().rsi_batch_create(arr, 1, 0, None, ctypes.byref(plan), ctypes.byref(ws),
                                          ctypes.byref(n))
        assert rc == -1
        return
    if bad == "no_points":
        cfg = copy.deepcopy(cfg)
        cfg["interfaces"][0]["n"] = 0
    if bad == "two_interfaces":
        cfg = copy.deepcopy(cfg)
        cfg["interfaces"].append(dict(cfg["interfaces"][0]))
        with pytest.raises(ValueError):
            rsi.Batch([cfg], allocate=False)
        return
    if bad == "fp64":
        shape = rsi.stage_struct(rsi.STAGE_RSI, "fp64", 1.0)
    with pytest.raises(rsi.RSIError):
        rsi.Batch([cfg], allocate=False, shape=shape)
