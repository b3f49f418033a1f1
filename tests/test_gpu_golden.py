"""Full-size chains on the GPU against stored FP64-oracle values.

tests/golden/<workload>.json holds the oracle's normalised image k phi / v0 at
1024 seeded pixels of each full-size workload, written by
tests/golden/make_golden.py (which calls only oracle/).  The GPU runs the
whole chain at full size, in the launch shapes bench.py times."""
import json
import os

import numpy as np
import pytest
import torch

from paper_2408_06765_gb300 import build, rsi
from paper_2408_06765_gb300 import workloads as W
from fieldcheck import assert_close

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-4  # FP32 pairs with a double-float phase


def workloads():
    out = {f"c2_{f / 1e6:g}MHz": W.c2_full_image(f) for f in W.C2_FREQS}
    out["c3_flat"] = W.c3_multilayer(curved=False)
    out["c3_curved"] = W.c3_multilayer(curved=True)
    return out


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load()


@pytest.mark.parametrize("name", sorted(workloads()))
def test_full_size_chain_matches_stored_oracle(name):
    path = os.path.join(HERE, f"{name}.json")
    if not os.path.exists(path):
        pytest.skip(f"no stored oracle values for {name}")
    rec = json.load(open(path))
    cfg = workloads()[name]
    img = rsi.run_chain(cfg).image
    torch.cuda.synchronize()
    rsi.sync_status()
    got = img.reshape(-1).cpu().numpy()[np.asarray(rec["pixels"])]
    want = np.asarray(rec["re"]) + 1j * np.asarray(rec["im"])
    assert_close(got, want, TOL, name)
