"""Write the stored expected values of the full-size parity tests.

Calls only the FP64 oracle (oracle/) and the workload descriptions.  For each
full-size workload it runs the whole oracle chain (piston -> every interface)
and evaluates the final stage on a seeded sample of image pixels, then stores
pixel indices and normalised values k phi / v0 as JSON text:

    python tests/golden/make_golden.py [name ...]

Workloads: c2 at 2.25, 5 and 10 MHz (2^16 x 2^18 points, 512^2 image), the
multilayer c3 workload, flat and curved (9 interfaces of 2^16 points), and the
two-medium image f1 (incident + reflected field above the interface,
transmitted field below, oracle.two_medium) and the ray-tracing model f2
(oracle.raytrace_image); the focused transducer f4 through both models.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2408_06765_gb300 import workloads as W  # noqa: E402

N_PIXELS = 1024


def cases():
    out = {f"c2_{f / 1e6:g}MHz": W.c2_full_image(f) for f in W.C2_FREQS}
    out["c3_flat"] = W.c3_multilayer(curved=False)
    out["c3_curved"] = W.c3_multilayer(curved=True)
    out["f1_5MHz"] = W.f1_two_medium()
    out["f2_5MHz"] = W.f2_ray_tracing()
    out["f4_chain_2.5MHz"] = W.f4_focused()
    out["f4_ray_2.5MHz"] = W.f4_focused()
    return out


def make_ray(name: str, cfg: dict):
    g = cfg["grid"]
    n_pix = int(g["nx"]) * int(g["nz"])
    rng = np.random.default_rng(1234)
    pix = np.sort(rng.choice(n_pix, N_PIXELS, replace=False))
    t0 = time.time()
    val = oracle.raytrace_image(cfg, pixels=pix)
    rec = {"workload": name, "source": "oracle.raytrace_image (FP64 CPU oracle), tests/golden/make_golden.py",
           "pixels": pix.tolist(), "re": val.real.tolist(), "im": val.imag.tolist(),
           "oracle_seconds": time.time() - t0}
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(rec, f)
    print(f"{name}: {time.time() - t0:.1f} s", flush=True)


def make_two_medium(name: str, cfg: dict):
    gw, gs = cfg["grid_water"], cfg["grid_solid"]
    n_pix = int(gw["nx"]) * (int(gw["nz"]) + int(gs["nz"]))
    rng = np.random.default_rng(1234)
    pix = np.sort(rng.choice(n_pix, N_PIXELS, replace=False))
    t0 = time.time()
    val = oracle.two_medium(cfg, pixels=pix)
    rec = {"workload": name, "source": "oracle.two_medium (FP64 CPU oracle), tests/golden/make_golden.py",
           "pixels": pix.tolist(), "re": val.real.tolist(), "im": val.imag.tolist(),
           "oracle_seconds": time.time() - t0}
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(rec, f)
    print(f"{name}: {time.time() - t0:.1f} s", flush=True)


def make(name: str, cfg: dict):
    g = cfg["grid"]
    n_pix = int(g["nx"]) * int(g["nz"])
    rng = np.random.default_rng(1234)
    pix = np.sort(rng.choice(n_pix, N_PIXELS, replace=False))
    grid = oracle.grid_points(g)
    targets = {k: grid[k][pix] for k in ("x", "y", "z")}
    t0 = time.time()
    phi, _ = oracle.chain(cfg, targets)
    k_last = oracle.wavenumber(cfg["freq"], cfg["media"][len(cfg["interfaces"])]["c"])
    val = (k_last / float(cfg["v0"])) * phi
    rec = {"workload": name, "source": "oracle.chain (FP64 CPU oracle), tests/golden/make_golden.py",
           "pixels": pix.tolist(), "re": val.real.tolist(), "im": val.imag.tolist(),
           "oracle_seconds": time.time() - t0}
    with open(os.path.join(HERE, f"{name}.json"), "w") as f:
        json.dump(rec, f)
    print(f"{name}: {time.time() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    want = sys.argv[1:]
    for name, cfg in cases().items():
        if not want or name in want:
            if "grid_water" in cfg:
                make_two_medium(name, cfg)
            elif name.startswith("f2") or name.startswith("f4_ray"):
                make_ray(name, cfg)
            else:
                make(name, cfg)
