"""The FMA-pipe sine and cosine of the stage kernels (csrc/sincos_poly.cuh):
the header is what its generator writes, and the polynomials, evaluated in
float32 with fused multiply-adds as the kernels evaluate them (including the
reduction t - rint(t) by adding and subtracting 1.5 * 2^23), stay within
7e-7 of sin(2 pi t) and cos(2 pi t) for phases of up to 2^20 turns
(the kernels' phases stay below a few hundred turns)."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_06765_gb300", "csrc")


def generator():
    spec = importlib.util.spec_from_file_location("gen_sincos_poly", os.path.join(CSRC, "gen_sincos_poly.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def f32(x):
    return np.asarray(x, np.float64).astype(np.float32)


def fma32(a, b, c):
    # a*b is exact in double for float inputs; one rounding to float after the add
    return f32(a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64))


def sincos_turns(t):
    t = f32(t)
    M = np.float32(12582912.0)
    r = f32(f32(t + M) - M)
    s = fma32(r, np.float32(-1.0), t)
    u = f32(s.astype(np.float64) * s)
    sc, cc = generator().coefficients()
    p = fma32(np.full_like(u, sc[5]), u, np.float32(sc[4]))
    for k in (3, 2, 1, 0):
        p = fma32(p, u, np.float32(sc[k]))
    sn = f32(p.astype(np.float64) * s)
    q = fma32(np.full_like(u, cc[6]), u, np.float32(cc[5]))
    for k in (4, 3, 2, 1, 0):
        q = fma32(q, u, np.float32(cc[k]))
    return sn, q, t


def test_header_is_the_generators_output():
    with open(os.path.join(CSRC, "sincos_poly.cuh")) as f:
        assert f.read() == generator().header()


def test_accuracy_over_one_turn():
    t = np.linspace(-0.5, 0.5, 400001)
    sn, cs, t32 = sincos_turns(t)
    x = 2 * np.pi * t32.astype(np.float64)
    assert np.max(np.abs(sn - np.sin(x))) < 7e-7
    assert np.max(np.abs(cs - np.cos(x))) < 7e-7
    assert np.all(np.abs(sn) <= 1.0 + 1e-6) and np.all(np.abs(cs) <= 1.0 + 1e-6)


def test_reduction_of_large_phases():
    rng = np.random.default_rng(0)
    for scale in (4.0, 300.0, 2.0 ** 20):
        t = rng.uniform(-scale, scale, 200000)
        sn, cs, t32 = sincos_turns(t)
        frac = t32.astype(np.float64) - np.rint(t32.astype(np.float64))  # exact in double
        x = 2 * np.pi * frac
        assert np.max(np.abs(sn - np.sin(x))) < 7e-7, scale
        assert np.max(np.abs(cs - np.cos(x))) < 7e-7, scale
