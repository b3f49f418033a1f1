"""Pins for the oracle's QMC generator and geometry maps (Sec. 2.3).

Each test ties the oracle to something other than itself: a published test
vector, the paper's Halton base-2 sequence, scipy's Sobol implementation,
the exact (0,m,2)-net property, or a closed-form area."""
import math

import numpy as np
import pytest

import oracle

GOLDEN = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def test_mix64_reproduces_splitmix64_stream():
    # SplitMix64 (Steele, Lea & Flood 2014) seeded with state 0: its first three
    # outputs as printed with the reference implementation.
    expected = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [oracle.mix64((k * GOLDEN) & M64) for k in (1, 2, 3)]
    assert got == expected


def _radical_inverse_base2(i: int) -> float:
    # Halton sequence H(n) for the prime n = 2 (Sec. 2.3, Eq. square_sampling)
    f, r = 0.5, 0.0
    while i:
        if i & 1:
            r += f
        i >>= 1
        f *= 0.5
    return r


def test_first_dimension_is_halton_base2():
    n = 4096
    su, _ = oracle.sobol(0, 0, n, scrambled=False)
    got = su.astype(np.float64) / 2.0**32
    want = np.array([_radical_inverse_base2(i) for i in range(n)])
    assert np.array_equal(got, want)


@pytest.mark.parametrize("m", [3, 6, 10])
def test_unscrambled_set_equals_scipy_sobol(m):
    qmc = pytest.importorskip("scipy.stats.qmc")
    su, sv = oracle.sobol(0, 0, 1 << m, scrambled=False)
    ours = sorted(zip((su / 2.0**32).tolist(), (sv / 2.0**32).tolist()))
    ref = qmc.Sobol(d=2, scramble=False).random_base2(m)
    theirs = sorted(map(tuple, ref.tolist()))
    assert ours == theirs


def _cells_exactly_once(su, sv, m):
    for a in range(m + 1):
        b = m - a
        cx = (su.astype(np.uint64) >> np.uint64(32 - a)) if a else np.zeros_like(su, np.uint64)
        cy = (sv.astype(np.uint64) >> np.uint64(32 - b)) if b else np.zeros_like(sv, np.uint64)
        cell = cx * np.uint64(1 << b) + cy
        counts = np.bincount(cell.astype(np.int64), minlength=1 << m)
        if not np.all(counts == 1):
            return False
    return True


@pytest.mark.parametrize("scrambled", [False, True])
@pytest.mark.parametrize("m,block", [(8, 0), (9, 3), (12, 1), (13, 0)])
def test_aligned_blocks_are_0m2_nets(scrambled, m, block):
    # Every aligned block of 2^m points of dims 1-2 is a (0,m,2)-net: each
    # elementary interval of area 2^-m holds exactly one point.  Nested
    # scrambling preserves this (Owen 1995).
    su, sv = oracle.sobol(5, 3, 1 << m, first=block << m, scrambled=scrambled)
    assert _cells_exactly_once(su, sv, m)


def test_scramble_is_nested():
    # output bit b depends only on input bits 0..b (from the top): inputs that
    # share a b-bit prefix give outputs that share it too, and the map is a
    # bijection of 32-bit words.
    key = oracle.scramble_key(0, 1, 0)
    rng = np.random.default_rng(1)
    for _ in range(200):
        x = int(rng.integers(0, 2**32))
        b = int(rng.integers(1, 32))
        flip = int(rng.integers(0, 2**(32 - b)))
        x2 = ((x >> (32 - b)) << (32 - b)) | flip
        y, y2 = oracle.owen(x, key), oracle.owen(x2, key)
        assert (y >> (32 - b)) == (y2 >> (32 - b))
    xs = np.arange(1 << 12, dtype=np.uint32) << np.uint32(20)
    ys = {oracle.owen(int(v), key) >> 20 for v in xs}
    assert len(ys) == 1 << 12


def test_scramble_is_uniform_over_seeds():
    # point 0 of the unscrambled sequence is (0, 0); scrambled over many seeds
    # it must look uniform on [0,1)^2 (Kolmogorov-Smirnov, both dims).
    stats = pytest.importorskip("scipy.stats")
    us, vs = [], []
    for seed in range(600):
        su, sv = oracle.sobol(seed, 0, 1, scrambled=True)
        us.append(su[0] / 2.0**32)
        vs.append(sv[0] / 2.0**32)
    assert stats.kstest(us, "uniform").pvalue > 1e-3
    assert stats.kstest(vs, "uniform").pvalue > 1e-3
    # different sets and dims get different keys
    keys = {oracle.scramble_key(0, s, d) for s in range(64) for d in (0, 1)}
    assert len(keys) == 128


def test_disk_map_geometry():
    a, tilt, c = 6.35e-3, math.radians(12.0), (1e-3, -2e-3, 3e-3)
    pts = oracle.make_points({"kind": "disk", "centre": c, "tilt": tilt, "a": a}, 0, 0, 5000)
    d = np.stack([pts["x"] - c[0], pts["y"] - c[1], pts["z"] - c[2]])
    nrm = np.array([math.sin(tilt), 0.0, math.cos(tilt)])
    assert np.allclose(nrm @ d, 0.0, atol=1e-18)  # points lie in the face plane
    assert np.all(np.linalg.norm(d, axis=0) <= a * (1 + 1e-15))
    assert np.allclose(np.stack([pts["nx"], pts["ny"], pts["nz"]]).T, nrm)
    assert math.isclose(pts["w"].sum(), math.pi * a * a, rel_tol=1e-12)
    # area-uniform radial law r = a sqrt(H) (Eq. circle_sampling): the fraction of
    # points inside radius a/2 is a quarter
    frac = np.mean(np.linalg.norm(d, axis=0) < a / 2)
    assert abs(frac - 0.25) < 2e-3


def test_rect_map_geometry():
    pts = oracle.make_points({"kind": "rect", "centre": (0.01, 0.0, 0.05), "wx": 0.06,
                              "wy": 0.04}, 0, 1, 4096)
    assert np.all(np.abs(pts["x"] - 0.01) < 0.03) and np.all(np.abs(pts["y"]) < 0.02)
    assert np.all(pts["z"] == 0.05) and np.all(pts["nz"] == 1.0)
    assert math.isclose(pts["w"].sum(), 0.06 * 0.04, rel_tol=1e-12)


def test_cylinder_map_geometry_and_area():
    R, wx, wy, c = 0.1, 0.06, 0.05, (0.002, 0.0, 0.03)
    pts = oracle.make_points({"kind": "cyl", "centre": c, "wx": wx, "wy": wy, "R": R}, 0, 4,
                             1 << 16)
    ax_z = c[2] + R
    rad = np.hypot(pts["x"] - c[0], pts["z"] - ax_z)
    assert np.allclose(rad, R, rtol=0, atol=1e-15)
    # normal points from the surface to the axis, unit length
    toward = np.stack([c[0] - pts["x"], np.zeros_like(rad), ax_z - pts["z"]]) / R
    assert np.allclose(np.stack([pts["nx"], pts["ny"], pts["nz"]]), toward, atol=1e-14)
    # sum of Jacobian weights -> lateral area of the cylindrical patch
    area = wy * R * 2.0 * math.asin(wx / (2.0 * R))
    assert math.isclose(pts["w"].sum(), area, rel_tol=2e-6)


def test_grid_is_cell_centred_row_major():
    g = {"x0": -0.02, "x1": 0.02, "nx": 4, "z0": 0.05, "z1": 0.09, "nz": 2, "y": 0.001}
    p = oracle.grid_points(g)
    assert np.allclose(p["x"][:4], [-0.015, -0.005, 0.005, 0.015])
    assert np.allclose(p["z"][::4], [0.06, 0.08])
    assert np.all(p["y"] == 0.001)
