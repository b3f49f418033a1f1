"""CUDA path vs the FP64 CPU oracle, through the C ABI.

Bars: Sobol integers, cell-order permutation and indices bit-exact; FP64
geometry to rounding; fields by relative L2 error <= 1e-5 (FP64 path) and
<= 1e-4 (FP32C path, double-float phase)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2408_06765_gb300 import build, rsi
from paper_2408_06765_gb300 import workloads as W
from fieldcheck import assert_close, max_rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-5, "fp32c": 1e-4}


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    return rsi.load()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def rel_l2(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def host_points(p: rsi.Points):
    torch.cuda.synchronize()
    out = {k: p.field(k).cpu().numpy() for k in ("X", "Y", "Z", "NX", "NY", "NZ", "W", "XH", "XL",
                                                  "YH", "YL", "ZH", "ZL")}
    out["IDX"], out["SU"], out["SV"] = u32(p.field("IDX")), u32(p.field("SU")), u32(p.field("SV"))
    return out


def expected_cells(n):
    """(block start, m) of the aligned power-of-two blocks of an n-point set."""
    blocks, start = [], 0
    for m in range(40, -1, -1):
        if n >> m & 1:
            blocks.append((start, m))
            start += 1 << m
    return blocks


def check_cell_order(idx, su, sv, n):
    for start, m in expected_cells(n):
        pos = np.arange(1 << m, dtype=np.uint64)
        a, b = (m + 1) // 2, m // 2
        cx = np.zeros_like(pos)
        cy = np.zeros_like(pos)
        for q in range(a):
            cx |= ((pos >> np.uint64(2 * q)) & np.uint64(1)) << np.uint64(q)
        for q in range(b):
            cy |= ((pos >> np.uint64(2 * q + 1)) & np.uint64(1)) << np.uint64(q)
        sl = slice(start, start + (1 << m))
        gx = (su[sl].astype(np.uint64) >> np.uint64(32 - a)) if a else np.zeros_like(pos)
        gy = (sv[sl].astype(np.uint64) >> np.uint64(32 - b)) if b else np.zeros_like(pos)
        assert np.array_equal(gx, cx) and np.array_equal(gy, cy)
        # the block holds exactly Sobol indices start .. start + 2^m - 1
        assert np.array_equal(np.sort(idx[sl]), np.arange(start, start + (1 << m)))


SURFACES = [
    {"kind": "disk", "centre": (1e-3, -2e-3, 0.5e-3), "tilt": math.radians(11.0), "a": 6.35e-3},
    {"kind": "rect", "centre": (2e-3, 0.0, 0.05), "wx": 0.06, "wy": 0.04},
    {"kind": "cyl", "centre": (0.0, 0.0, 0.03), "wx": 0.06, "wy": 0.06, "R": 0.1},
]


@pytest.mark.parametrize("surf", SURFACES, ids=lambda s: s["kind"])
@pytest.mark.parametrize("n,seed,set_id", [(1, 0, 0), (7, 3, 2), (256, 0, 1), (1000, 5, 9),
                                          (4096, 0, 1), (65536 + 300, 1, 4)])
def test_qmc_points_bit_exact(surf, n, seed, set_id):
    p = host_points(rsi.make_qmc_points(surf, seed, set_id, n))
    idx = p["IDX"]
    assert np.array_equal(np.sort(idx), np.arange(n, dtype=np.uint32))
    su_o, sv_o = oracle.sobol(seed, set_id, n)
    assert np.array_equal(p["SU"], su_o[idx]) and np.array_equal(p["SV"], sv_o[idx])
    check_cell_order(idx, p["SU"], p["SV"], n)
    ref = oracle.map_points(surf, su_o, sv_o)
    # FP64 geometry: a few ulps of the largest term entering each coordinate
    extent = sum(abs(c) for c in surf["centre"]) + 2 * max(surf.get(k, 0.0) for k in ("a", "wx", "wy", "R"))
    for key in ("x", "y", "z", "nx", "ny", "nz", "w"):
        got, want = p[key.upper()], ref[key][idx]
        scale = extent if key in ("x", "y", "z") else float(np.max(np.abs(want)))
        assert np.max(np.abs(got - want)) <= 8 * 2.0**-52 * scale + 1e-300, key
    for c in ("X", "Y", "Z"):
        assert np.array_equal(p[c + "H"], p[c].astype(np.float32))
        assert np.array_equal(p[c + "L"], (p[c] - p[c + "H"].astype(np.float64)).astype(np.float32))


def test_unscrambled_points_are_plain_sobol():
    p = host_points(rsi.make_qmc_points(SURFACES[1], 0, 0, 1 << 10, scramble=False))
    su_o, sv_o = oracle.sobol(0, 0, 1 << 10, scrambled=False)
    assert np.array_equal(p["SU"], su_o[p["IDX"]]) and np.array_equal(p["SV"], sv_o[p["IDX"]])


def test_grid_points():
    g = {"x0": -0.015, "x1": 0.017, "nx": 37, "z0": 0.03, "z1": 0.055, "nz": 29, "y": 1e-3}
    p = host_points(rsi.grid_points(g))
    ref = oracle.grid_points(g)
    for key in ("x", "y", "z"):
        assert np.max(np.abs(p[key.upper()] - ref[key])) <= 1e-17
    assert np.array_equal(p["IDX"], np.arange(37 * 29, dtype=np.uint32))


# ---------------------------------------------------------------------------
# chains
# ---------------------------------------------------------------------------
def chain_parity(cfg, tol, stage_opts=None):
    res = rsi.run_chain(cfg, keep=True, stage_opts=stage_opts)
    torch.cuda.synchronize()
    rsi.sync_status()
    ref_phi, ref_kept = oracle.chain(cfg, keep=True)
    errs, worst = [], []
    for (gpts, gphi), (_, ophi) in zip(res.ifaces, ref_kept):
        idx = u32(gpts.field("IDX"))
        errs.append(rel_l2(gphi.cpu().numpy(), ophi[idx]))
        worst.append(max_rel(gphi.cpu().numpy(), ophi[idx]))
    g = cfg["grid"]
    k_last = oracle.wavenumber(cfg["freq"], cfg["media"][len(cfg["interfaces"])]["c"])
    img_ref = (k_last / cfg["v0"]) * ref_phi.reshape(g["nz"], g["nx"])
    errs.append(rel_l2(res.image.cpu().numpy(), img_ref))
    worst.append(max_rel(res.image.cpu().numpy(), img_ref))
    assert max(errs) <= tol, errs
    assert max(worst) <= 10 * tol, worst  # no error confined to a few pixels
    return errs, res


def test_small_ragged_fp64():
    errs, _ = chain_parity(W.small_ragged("fp64"), TOL["fp64"])
    assert max(errs) < 1e-11  # FP64 end to end: rounding-level agreement


@pytest.mark.parametrize("freq", W.C2_FREQS)
def test_small_ragged_fp32c(freq):
    chain_parity(W.small_ragged("fp32c", freq=freq), TOL["fp32c"])


@pytest.mark.parametrize("tilt_deg", [10.0, 20.0])
def test_small_ragged_tilted_and_postcritical(tilt_deg):
    # 20 deg is past the water -> steel critical angle (14.5 deg): complex T12
    cfg = W.small_ragged("fp32c", tilt=math.radians(tilt_deg))
    chain_parity(cfg, TOL["fp32c"])
    chain_parity(dict(cfg, precision="fp64"), TOL["fp64"])


def test_c1_plain_fp64():
    errs, _ = chain_parity(W.c1_plain_fp64(), TOL["fp64"])
    assert max(errs) < 1e-11


@pytest.mark.parametrize("curved", [False, True])
def test_multilayer_reduced_counts(curved):
    cfg = W.c3_multilayer(curved=curved, n_per_surface=1 << 11)
    chain_parity(cfg, TOL["fp32c"])


@pytest.mark.parametrize("opts", [
    {"tile": 32, "tpt": 2, "splits": 1, "variant": 1},
    {"tile": 64, "tpt": 4, "splits": 3, "variant": 2},
    {"tile": 128, "tpt": 2, "splits": 0, "variant": 2},
    {"tile": 512, "tpt": 4, "splits": 2, "variant": 1},
    {"tile": 32, "tpt": 2, "splits": 1, "variant": 3},
    {"tile": 256, "tpt": 4, "splits": 0, "variant": 3},
    {"tile": 128, "tpt": 2, "splits": 5, "variant": 3},
    {"tile": 64, "tpt": 1, "splits": 2, "variant": 3},
    {"tile": 256, "tpt": 1, "splits": 0, "variant": 1},
    {"tile": 32, "tpt": 1, "splits": 1, "variant": 2},
])
def test_launch_shapes_agree(opts):
    cfg = W.small_ragged("fp32c", freq=7.5e6)
    errs, res = chain_parity(cfg, TOL["fp32c"], stage_opts=opts)
    base = rsi.run_chain(cfg).image
    assert rel_l2(res.image.cpu().numpy(), base.cpu().numpy()) < 2e-5


@pytest.mark.parametrize("curved", [False, True])
def test_packed_variant_multilayer(curved):
    # two sources per f32x2 instruction, with per-point normals on the curved stack
    cfg = W.c3_multilayer(curved=curved, n_per_surface=1 << 11)
    chain_parity(cfg, TOL["fp32c"], stage_opts={"variant": 3})


@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32c_packed"])
def test_coincident_targets_contribute_nothing(prec):
    # a surface propagated onto its own points: every target coincides with one
    # source, whose term is dropped (both sides)
    rng = np.random.default_rng(0)
    k = 2 * math.pi * 2e6 / 1480.0
    sig = rng.normal(size=700) + 1j * rng.normal(size=700)
    sig_d = torch.tensor(sig, device="cuda")
    # flat patch: every chord lies in the plane, cos(theta) = 0, the RSI field is 0
    flat = rsi.make_qmc_points({"kind": "rect", "centre": (0.0, 0.0, 0.02), "wx": 0.02, "wy": 0.02},
                               0, 1, 700)
    var = 3 if prec == "fp32c_packed" else 0
    prec = "fp32c" if prec == "fp32c_packed" else prec
    out = rsi.propagate_stage(rsi.stage_struct(rsi.STAGE_RSI, prec, k, normals=rsi.NORMALS_Z, variant=var),
                              flat, sig_d, flat)
    rsi.sync_status()
    hp = host_points(flat)
    src = {"x": hp["X"], "y": hp["Y"], "z": hp["Z"], "nx": hp["NX"], "ny": hp["NY"], "nz": hp["NZ"],
           "w": hp["W"]}
    assert np.all(out.cpu().numpy() == 0) and np.all(oracle.rsi_field(src, sig, src, k) == 0)
    out = rsi.propagate_stage(rsi.stage_struct(rsi.STAGE_PISTON, prec, k, variant=var), flat, None, flat)
    rsi.sync_status()
    ref = oracle.piston_field(src, src, k)
    assert np.all(np.isfinite(out.cpu().numpy()))
    assert_close(out.cpu().numpy(), ref, TOL[prec])
    # curved surface: chords are not normal to the surface normals
    cyl = rsi.make_qmc_points({"kind": "cyl", "centre": (0.0, 0.0, 0.02), "wx": 0.03, "wy": 0.03,
                               "R": 0.02}, 0, 2, 700)
    out = rsi.propagate_stage(rsi.stage_struct(rsi.STAGE_RSI, prec, k, normals=rsi.NORMALS_POINTS, variant=var),
                              cyl, sig_d, cyl)
    rsi.sync_status()
    hp = host_points(cyl)
    src = {"x": hp["X"], "y": hp["Y"], "z": hp["Z"], "nx": hp["NX"], "ny": hp["NY"], "nz": hp["NZ"],
           "w": hp["W"]}
    ref = oracle.rsi_field(src, sig, src, k)
    assert np.all(np.isfinite(out.cpu().numpy()))
    assert_close(out.cpu().numpy(), ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_single_source_single_target(prec):
    pist = rsi.make_qmc_points({"kind": "disk", "centre": (0, 0, 0), "a": 5e-3}, 0, 0, 1)
    tgt = rsi.grid_points({"x0": 1e-3, "x1": 1e-3, "nx": 1, "z0": 0.04, "z1": 0.04, "nz": 1})
    k = 2 * math.pi * 5e6 / 1480.0
    out = rsi.propagate_stage(rsi.stage_struct(rsi.STAGE_PISTON, prec, k, 2.0), pist, None, tgt)
    hp = host_points(pist)
    ref = oracle.piston_field({"x": hp["X"], "y": hp["Y"], "z": hp["Z"], "w": hp["W"]},
                              {"x": np.array([1e-3]), "y": np.zeros(1), "z": np.array([0.04])}, k, 2.0)
    assert_close(out.cpu().numpy(), ref, TOL[prec])


def test_status_word_is_clean():
    rsi.sync_status()


# ---------------------------------------------------------------------------
# full-size c2 geometry, sampled outputs (launch shapes of the bench)
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_c2_full_size_sampled():
    cfg = W.c2_full_image(10e6)
    res = rsi.run_chain(cfg, keep=True)
    torch.cuda.synchronize()
    rsi.sync_status()
    (gif, gphi), = res.ifaces
    idx = u32(gif.field("IDX"))
    rng = np.random.default_rng(11)
    # stage 1: all 2^16 piston points onto 1024 sampled interface points
    pc = cfg["piston"]
    o_pist = oracle.make_points(dict(pc, kind="disk"), 0, 0, pc["n"])
    o_if = oracle.make_points(cfg["interfaces"][0], 0, 1, cfg["interfaces"][0]["n"])
    slots = rng.choice(gif.n, 1024, replace=False)
    tg = {key: o_if[key][idx[slots]] for key in ("x", "y", "z")}
    k1 = oracle.wavenumber(cfg["freq"], 1480.0)
    ref1 = oracle.piston_field(o_pist, tg, k1)
    assert_close(gphi.cpu().numpy()[slots], ref1, TOL["fp32c"])
    # stage 2 at full size with an oracle-side source density (a tilted
    # Gaussian beam on the 2^18 interface points), sampled on 2048 pixels
    k2 = oracle.wavenumber(cfg["freq"], 5900.0)
    sig_o = np.exp(-(o_if["x"] ** 2 + o_if["y"] ** 2) / (12e-3) ** 2
                   + 1j * k2 * math.sin(math.radians(5.0)) * o_if["x"])
    grid = rsi.grid_points(cfg["grid"])
    st = rsi.stage_struct(rsi.STAGE_RSI, "fp32c", k2, normals=rsi.NORMALS_Z)
    out = rsi.propagate_stage(st, gif, torch.tensor(sig_o[idx], device="cuda"), grid)
    rsi.sync_status()
    pix = rng.choice(grid.n, 2048, replace=False)
    og = oracle.grid_points(cfg["grid"])
    ref2 = oracle.rsi_field(o_if, sig_o, {key: og[key][pix] for key in ("x", "y", "z")}, k2)
    assert_close(out.cpu().numpy()[pix], ref2, TOL["fp32c"])
