"""Pins of the oracle's ray-tracing model (Sec. 2.2): the solved ray path
against Snell's law, geometric closure and Fermat's principle; the spreading
factor of Eq. transmitted_ray_tracing against the ray-tube Jacobian taken by
finite differences; reductions to the direct piston field (one medium) and
to T12 times it (a density step); and agreement with the RSI chain, the
paper's other model of the same field."""
import math

import numpy as np
import pytest

import oracle
from test_oracle_fields import disk_quadrature, plane_quadrature, points

WATER = {"rho": 1000.0, "c": 1480.0}
STEEL = {"rho": 7800.0, "c": 5900.0}


def rho_of(theta1, h1, h2, c1, c2):
    """Horizontal reach of the ray leaving at angle theta1 (Snell at the plane)."""
    s2 = c2 / c1 * np.sin(theta1)
    return h1 * np.tan(theta1) + h2 * s2 / np.sqrt(1.0 - s2 * s2)


@pytest.mark.parametrize("h1,h2,rho", [(0.05, 0.01, 0.02), (0.03, 0.04, 0.0), (0.05, 0.002, 0.045),
                                       (0.01, 0.06, 0.005), (0.05, 0.03, 0.08)])
def test_ray_path_obeys_snell_closure_and_fermat(h1, h2, rho):
    c1, c2 = WATER["c"], STEEL["c"]
    p = oracle.ray_path(h1, h2, rho, c1, c2)
    s1, s2 = math.sqrt(1 - p["cos1"] ** 2), math.sqrt(1 - p["cos2"] ** 2)
    # Eq. root_searching (sines rebuilt from the cosines: ~1e-13 relative at small angles)
    assert abs(s1 / c1 - s2 / c2) <= 1e-11 * max(s1 / c1, 1e-300) + 1e-20
    reach = h1 * s1 / p["cos1"] + h2 * s2 / p["cos2"]  # geometric closure, Eq. ray_tracing
    assert abs(reach - rho) <= 1e-12 * max(rho, h1 + h2)
    # Fermat: the crossing point minimises the travel time D1/c1 + D2/c2
    t = np.linspace(0.0, rho, 200001) if rho > 0 else np.zeros(1)
    times = np.sqrt(h1 ** 2 + t ** 2) / c1 + np.sqrt(h2 ** 2 + (rho - t) ** 2) / c2
    solved = p["D1"] / c1 + p["D2"] / c2
    assert solved <= times.min() * (1 + 1e-13)
    assert solved >= times.min() * (1 - 1e-9)


@pytest.mark.parametrize("theta1_deg,h1,h2", [(3.0, 0.05, 0.02), (8.0, 0.03, 0.01), (13.0, 0.05, 0.005),
                                              (10.0, 0.02, 0.06)])
def test_spreading_factor_is_the_ray_tube_jacobian(theta1_deg, h1, h2):
    # For one transducer point and one field point the ray-tracing sum is a
    # single term, so its magnitude gives the denominator of Eq.
    # transmitted_ray_tracing.  A ray tube from a point source spreads by
    # (rho / sin a1) in the azimuthal direction and by cos a1 d(rho)/d(a1) in
    # the plane of incidence; their product must equal that denominator.
    c1, c2 = WATER["c"], STEEL["c"]
    th = math.radians(theta1_deg)
    rho = float(rho_of(th, h1, h2, c1, c2))
    d = 1e-6
    drho = float((rho_of(th + d, h1, h2, c1, c2) - rho_of(th - d, h1, h2, c1, c2)) / (2 * d))
    jac = (rho / math.sin(th)) * (math.cos(th) * drho)
    src = {"x": np.zeros(1), "y": np.zeros(1), "z": np.array([-h1]), "w": np.ones(1)}
    tgt = points([[rho, 0.0, h2]])
    k1 = 2 * np.pi * 5e6 / c1
    phi = oracle.raytrace_field(src, tgt, WATER, STEEL, 0.0, k1, k1 * c1 / c2)
    p = oracle.ray_path(h1, h2, rho, c1, c2)
    T = oracle.T12(WATER["rho"], c1, STEEL["rho"], c2, p["cos1"], p["cos2"])
    den = (abs(T) / (2 * np.pi) / abs(phi[0])) ** 2
    assert den == pytest.approx(jac, rel=1e-7)


def test_one_medium_rays_are_straight_and_give_the_direct_field():
    a, k = 3e-3, 2 * np.pi * 3e6 / 1480.0
    pist = disk_quadrature(a, n_r=12, n_t=36, tilt=0.15)
    tq = np.array([[0, 0, 20e-3], [4e-3, -1e-3, 35e-3], [-6e-3, 2e-3, 12e-3]])
    got = oracle.raytrace_field(pist, points(tq), WATER, WATER, 8e-3, k, k)
    want = oracle.piston_field(pist, points(tq), k)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-12


def test_density_step_scales_by_T():
    # equal speeds: straight rays at every angle, T12 = 2 rho1 / (rho1 + rho2)
    a, k = 3e-3, 2 * np.pi * 3e6 / 1480.0
    pist = disk_quadrature(a, n_r=12, n_t=36)
    heavy = {"rho": 3000.0, "c": 1480.0}
    tq = np.array([[0, 0, 20e-3], [5e-3, 0, 30e-3]])
    got = oracle.raytrace_field(pist, points(tq), WATER, heavy, 10e-3, k, k)
    want = 0.5 * oracle.piston_field(pist, points(tq), k)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-12


def test_ray_tracing_agrees_with_the_rsi_chain():
    # The paper's two models of the transmitted field (Sec. 2.1 and 2.2) agree
    # away from the interface at high frequency.  Both sums use Gauss-Legendre
    # rules here, so the difference is the models' own (a few per cent).
    a, f = 3e-3, 5e6
    c1, c2 = WATER["c"], STEEL["c"]
    k1, k2 = 2 * np.pi * f / c1, 2 * np.pi * f / c2
    zi = 12e-3
    pist = disk_quadrature(a, n_r=24, n_t=72)
    iface = plane_quadrature(0.012, 0.2e-3, 8, z0=zi, window=(0.008, 0.012))
    phi_i = oracle.piston_field(pist, iface, k1)
    sigma, _ = oracle.transmit(iface, phi_i, WATER, STEEL, 0.0, "global")
    tq = np.array([[0, 0, zi + 10e-3], [0, 0, zi + 20e-3], [1e-3, 0, zi + 15e-3]])
    rsi = oracle.rsi_field(iface, sigma, points(tq), k2)
    ray = oracle.raytrace_field(pist, points(tq), WATER, STEEL, zi, k1, k2)
    assert np.max(np.abs(ray - rsi) / np.abs(rsi)) < 0.05
