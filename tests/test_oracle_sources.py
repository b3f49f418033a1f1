"""Pins of the oracle's f3/f4 point sets: the Halton sequence of Sec. 2.3
(textbook first values, plain-Python radical inverses, stratification), the
focused transducer's spherical cap (points on the sphere, normals to the
centre of curvature, area, O'Neil's on-axis closed form) and the Gaussian
apodisation of the face (weights, on-axis field against an adaptive 1-D
quadrature)."""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

import oracle

MM = 1e-3


def radical_inverse(i: int, base: int) -> Fraction:
    f, scale = Fraction(0), Fraction(1, base)
    while i:
        f += (i % base) * scale
        i //= base
        scale /= base
    return f


def test_halton_first_values():
    su, sv = oracle.halton(9)
    want2 = [Fraction(1, 2), Fraction(1, 4), Fraction(3, 4), Fraction(1, 8), Fraction(5, 8), Fraction(3, 8),
             Fraction(7, 8), Fraction(1, 16), Fraction(9, 16)]
    want3 = [Fraction(1, 3), Fraction(2, 3), Fraction(1, 9), Fraction(4, 9), Fraction(7, 9), Fraction(2, 9),
             Fraction(5, 9), Fraction(8, 9), Fraction(1, 27)]
    assert [Fraction(int(x), 2 ** 32) for x in su] == want2
    assert [Fraction(int(y), 3 ** 20) for y in sv] == want3


def test_halton_matches_plain_radical_inverses():
    rng = np.random.default_rng(0)
    for first in [0, 1000, int(rng.integers(0, 2 ** 31 - 100))]:
        su, sv = oracle.halton(40, first)
        for q in range(40):
            i = first + q + 1
            assert Fraction(int(su[q]), 2 ** 32) == radical_inverse(i, 2)
            assert Fraction(int(sv[q]), 3 ** 20) == radical_inverse(i, 3)


def test_halton_stratifies_both_bases():
    # the first b^k points of the base-b van der Corput sequence (indices 1 .. b^k
    # here, a rotation of 0 .. b^k - 1) hit every interval [j / b^k, (j+1) / b^k) once
    su, sv = oracle.halton(3 ** 7)
    cells3 = np.asarray(sv, np.uint64) // (3 ** 13)
    assert sorted(cells3.tolist()) == list(range(3 ** 7))
    su2, _ = oracle.halton(2 ** 11)
    assert sorted((np.asarray(su2, np.uint64) >> 21).tolist()) == list(range(2 ** 11))


def cap_surface(tilt=0.0, apod=0.0, seq="sobol"):
    return {"kind": "cap", "centre": (1 * MM, -2 * MM, 3 * MM), "tilt": tilt, "a": 6.35 * MM, "R": 33 * MM,
            "apod": apod, "sequence": seq}


@pytest.mark.parametrize("tilt", [0.0, 0.3])
@pytest.mark.parametrize("seq", ["sobol", "halton"])
def test_cap_points_lie_on_the_sphere(tilt, seq):
    s = cap_surface(tilt, seq=seq)
    p = oracle.make_points(s, 0, 5, 5000)
    R, a = s["R"], s["a"]
    c = np.array(s["centre"])
    axis = np.array([math.sin(tilt), 0.0, math.cos(tilt)])
    C = c + R * axis  # centre of curvature
    xyz = np.stack([p["x"], p["y"], p["z"]], 1)
    assert np.max(np.abs(np.linalg.norm(xyz - C, axis=1) - R)) < 1e-15 * R * 8
    n = np.stack([p["nx"], p["ny"], p["nz"]], 1)
    assert np.max(np.abs(np.linalg.norm(n, axis=1) - 1)) < 1e-15 * 8
    assert np.max(np.abs(n - (C - xyz) / R)) < 1e-15 * 8
    off = (xyz - c) - np.outer((xyz - c) @ axis, axis)
    assert np.max(np.linalg.norm(off, axis=1)) <= a * (1 + 1e-15)
    area = 2 * math.pi * R * (R - math.sqrt(R * R - a * a))
    assert abs(p["w"].sum() - area) < 2e-3 * area


def oneil_on_axis(z, a, R, k, v0=1.0):
    """O'Neil (1949): Eq. incident_field over a spherical cap on its axis,
    -(v0 R / (i k (R - z))) (e^{ik r_rim} - e^{ikz}), apex at z = 0."""
    r_rim = np.sqrt(R * R + (R - z) ** 2 - 2 * R * (R - z) * math.sqrt(1 - (a / R) ** 2))
    return -(v0 * R / (1j * k * (R - z))) * (np.exp(1j * k * r_rim) - np.exp(1j * k * z))


def test_cap_on_axis_field_is_oneils_closed_form():
    a, R, k = 6.35 * MM, 33 * MM, 2 * np.pi * 2.5e6 / 1480.0
    z = np.array([5 * MM, 20 * MM, 29 * MM, 45 * MM])
    # Gauss-Legendre in the polar angle about the centre of curvature x trapezoid
    amax = math.asin(a / R)
    xg, wg = np.polynomial.legendre.leggauss(96)
    al, wa = 0.5 * amax * (xg + 1), 0.5 * amax * wg
    ps = 2 * np.pi * (np.arange(128) + 0.5) / 128
    A, P = np.meshgrid(al, ps, indexing="ij")
    W = np.outer(wa * R * R * np.sin(al), np.full(128, 2 * np.pi / 128))
    gl = {"x": (R * np.sin(A) * np.cos(P)).ravel(), "y": (R * np.sin(A) * np.sin(P)).ravel(),
          "z": (R - R * np.cos(A)).ravel(), "w": W.ravel()}
    tq = {"x": 0 * z, "y": 0 * z, "z": z}
    want = oneil_on_axis(z, a, R, k)
    assert np.max(np.abs(oracle.piston_field(gl, tq, k) - want) / np.abs(want)) < 1e-10
    # the oracle's QMC cap reproduces it to QMC accuracy
    s = dict(cap_surface(), centre=(0.0, 0.0, 0.0))
    qmc = oracle.make_points(s, 0, 1, 1 << 15)
    assert np.max(np.abs(oracle.piston_field(qmc, tq, k) - want) / np.abs(want)) < 3e-3


def test_apodised_disk_weights_and_on_axis_field():
    a, g, k = 6.35 * MM, 4 * MM, 2 * np.pi * 2.5e6 / 1480.0
    s = {"kind": "disk", "centre": (0.0, 0.0, 0.0), "tilt": 0.0, "a": a, "apod": g}
    p = oracle.make_points(s, 0, 2, 1 << 15)
    u = dict(s, apod=0.0)
    q = oracle.make_points(u, 0, 2, 1 << 15)
    r2 = p["x"] ** 2 + p["y"] ** 2
    assert np.allclose(p["w"], q["w"] * np.exp(-r2 / g ** 2), rtol=1e-14, atol=0)
    # on-axis: -(v0 / 2 pi) int_0^a int_0^2pi e^{-r^2/g^2} e^{ik rho} / rho r dr dtheta, rho = sqrt(z^2 + r^2)
    for z in (10 * MM, 40 * MM):
        f = lambda r, part: (np.exp(-(r / g) ** 2) * np.exp(1j * k * math.hypot(z, r)) / math.hypot(z, r) * r)
        re = integrate.quad(lambda r: f(r, 0).real, 0, a, epsabs=0, epsrel=1e-12, limit=400)[0]
        im = integrate.quad(lambda r: f(r, 0).imag, 0, a, epsabs=0, epsrel=1e-12, limit=400)[0]
        want = -(re + 1j * im)  # -(v0/2pi) * 2pi * radial integral
        got = oracle.piston_field(p, {"x": np.zeros(1), "y": np.zeros(1), "z": np.array([z])}, k)[0]
        assert abs(got - want) < 3e-3 * abs(want)
