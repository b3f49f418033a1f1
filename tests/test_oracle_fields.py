"""Pins for the oracle's stage sums and interface coefficients (Sec. 2.1).

The stage functions take arbitrary weighted points, so each is checked with
deterministic Gauss-Legendre quadratures against results the mathematics
fixes: the closed-form on-axis field of a circular piston, the first
Rayleigh-Sommerfeld solution reproducing an outgoing spherical wave, and the
matched-impedance chain reproducing the single-medium field.  Interface
coefficients are checked against the reflection-coefficient identity and
energy conservation; QMC convergence against the closed form."""
import math

import numpy as np
import pytest

import oracle


# ---------------------------------------------------------------------------
# deterministic quadratures
# ---------------------------------------------------------------------------
def disk_quadrature(a, n_r=64, n_t=64, centre=(0.0, 0.0, 0.0), tilt=0.0):
    """Gauss-Legendre in r (weight r dr) x trapezoid in theta on a tilted disk."""
    xr, wr = np.polynomial.legendre.leggauss(n_r)
    r = 0.5 * a * (xr + 1.0)
    wr = 0.5 * a * wr * r
    th = 2.0 * np.pi * (np.arange(n_t) + 0.5) / n_t
    R, TH = np.meshgrid(r, th, indexing="ij")
    W = np.outer(wr, np.full(n_t, 2.0 * np.pi / n_t))
    l1, l2 = (R * np.cos(TH)).ravel(), (R * np.sin(TH)).ravel()
    ct, st = math.cos(tilt), math.sin(tilt)
    n = l1.size
    return {"x": centre[0] + l1 * ct, "y": centre[1] + l2, "z": centre[2] - l1 * st,
            "nx": np.full(n, st), "ny": np.zeros(n), "nz": np.full(n, ct), "w": W.ravel()}


def smooth_window(rho, l1, l2):
    """1 for rho <= l1, 0 for rho >= l2, C-infinity in between."""
    t = np.clip((l2 - rho) / (l2 - l1), 0.0, 1.0)
    f = lambda s: np.where(s > 0, np.exp(-1.0 / np.maximum(s, 1e-300)), 0.0)
    return f(t) / (f(t) + f(1.0 - t))


def plane_quadrature(half, panel, order, z0=0.0, window=None, cx=0.0):
    """Composite Gauss-Legendre on [-half, half]^2 in the plane z = z0, normal +z,
    optionally multiplied by a smooth radial window (l1, l2)."""
    xg, wg = np.polynomial.legendre.leggauss(order)
    edges = np.arange(-half, half + 1e-15, panel)
    xs = np.concatenate([0.5 * (b - a) * xg + 0.5 * (a + b) for a, b in zip(edges[:-1], edges[1:])])
    ws = np.concatenate([0.5 * (b - a) * wg for a, b in zip(edges[:-1], edges[1:])])
    X, Y = np.meshgrid(xs + cx, xs, indexing="ij")
    W = np.outer(ws, ws)
    if window is not None:
        W = W * smooth_window(np.hypot(X - cx, Y), *window)
    keep = W.ravel() != 0.0
    n = int(keep.sum())
    return {"x": X.ravel()[keep], "y": Y.ravel()[keep], "z": np.full(n, z0),
            "nx": np.zeros(n), "ny": np.zeros(n), "nz": np.ones(n), "w": W.ravel()[keep]}


def points(xyz):
    xyz = np.atleast_2d(np.asarray(xyz, np.float64))
    return {"x": xyz[:, 0], "y": xyz[:, 1], "z": xyz[:, 2]}


def piston_on_axis(z, a, k, v0=1.0):
    """Integral of Eq. incident_field over a disk of radius a on its axis:
    phi = (v0 / (i k)) (e^{ikz} - e^{ik sqrt(z^2 + a^2)})."""
    return v0 / (1j * k) * (np.exp(1j * k * z) - np.exp(1j * k * np.sqrt(z * z + a * a)))


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# ---------------------------------------------------------------------------
# piston stage (Eq. incident_field)
# ---------------------------------------------------------------------------
def test_piston_on_axis_closed_form():
    a, k = 6.35e-3, 2 * np.pi * 2.5e6 / 1480.0
    z = np.array([2e-3, 10e-3, 35e-3, 100e-3])
    got = oracle.piston_field(disk_quadrature(a), points(np.stack([0 * z, 0 * z, z], 1)), k, 1.0)
    assert rel(got, piston_on_axis(z, a, k)) < 1e-10
    # |k phi / v0| = 2 |sin(k (sqrt(z^2 + a^2) - z) / 2)|  (normalisation of Sec. 3)
    assert np.allclose(np.abs(k * got), 2 * np.abs(np.sin(k * (np.hypot(z, a) - z) / 2)),
                       rtol=1e-9)


def test_piston_on_tilted_axis():
    a, k, tilt, c = 5e-3, 2 * np.pi * 5e6 / 1480.0, math.radians(17.0), (2e-3, 1e-3, -1e-3)
    axis = np.array([math.sin(tilt), 0.0, math.cos(tilt)])
    d = np.array([3e-3, 20e-3, 60e-3])
    tgt = points(np.array(c)[None, :] + d[:, None] * axis[None, :])
    got = oracle.piston_field(disk_quadrature(a, centre=c, tilt=tilt), tgt, k, 2.0)
    assert rel(got, piston_on_axis(d, a, k, 2.0)) < 1e-10


def test_piston_qmc_points_converge_to_closed_form():
    a, k = 6.35e-3, 2 * np.pi * 5e6 / 1480.0
    z = np.array([30e-3, 60e-3, 120e-3])
    tgt = points(np.stack([0 * z, 0 * z, z], 1))
    pts = oracle.make_points({"kind": "disk", "centre": (0, 0, 0), "tilt": 0.0, "a": a}, 0, 0,
                             1 << 16)
    assert rel(oracle.piston_field(pts, tgt, k), piston_on_axis(z, a, k)) < 2e-4


def test_qmc_error_decays_faster_than_mc_rate():
    # Sec. 2.3: low-discrepancy sampling converges faster than N^-1/2.
    a, k = 6.35e-3, 2 * np.pi * 5e6 / 1480.0
    z = np.array([20e-3, 45e-3, 90e-3])
    tgt = points(np.stack([0 * z, 0 * z, z], 1))
    exact = piston_on_axis(z, a, k)
    ns = [1 << m for m in range(8, 17, 2)]
    errs = []
    for n in ns:
        e2 = []
        for seed in range(6):
            pts = oracle.make_points({"kind": "disk", "centre": (0, 0, 0), "tilt": 0.0, "a": a},
                                     seed, 0, n)
            e2.append(rel(oracle.piston_field(pts, tgt, k), exact) ** 2)
        errs.append(math.sqrt(np.mean(e2)))
    slope = np.polyfit(np.log(ns), np.log(errs), 1)[0]
    assert slope < -0.8, (slope, errs)


# ---------------------------------------------------------------------------
# RSI stage (Eq. rayleigh_sommerfeld)
# ---------------------------------------------------------------------------
def test_rsi_reproduces_outgoing_spherical_wave():
    # A point source at depth -d radiates e^{ikR}/R; Eq. rayleigh_sommerfeld over
    # the plane z = 0 (normal toward the observation side) must reproduce it at
    # z > 0 -- the first Rayleigh-Sommerfeld solution is exact for outgoing fields.
    k = 2 * np.pi / 1e-3
    d = 4e-3
    src = plane_quadrature(0.03, 0.75e-3, 12, window=(0.012, 0.03))
    R = np.sqrt(src["x"] ** 2 + src["y"] ** 2 + d * d)
    sigma = np.exp(1j * k * R) / R
    tq = np.array([[0, 0, 5e-3], [3e-3, 2e-3, 10e-3], [0, 0, 0.4e-3], [1e-3, 0, 1.5e-3]])
    got = oracle.rsi_field(src, sigma, points(tq), k)
    Rq = np.sqrt(tq[:, 0] ** 2 + tq[:, 1] ** 2 + (tq[:, 2] + d) ** 2)
    want = np.exp(1j * k * Rq) / Rq
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-6


def test_matched_impedance_chain_reproduces_direct_field():
    # Identical media: T12 = 1, and piston -> interface -> field must equal the
    # direct piston field beyond the interface (Sec. 3.1 display convention).
    a, k, zi = 3e-3, 2 * np.pi / 2e-3, 10e-3
    pist = disk_quadrature(a, n_r=16, n_t=48)
    iface = plane_quadrature(0.04, 1.6e-3, 12, z0=zi, window=(0.016, 0.04))
    phi_i = oracle.piston_field(pist, iface, k)
    water = {"rho": 1000.0, "c": 1480.0}
    sigma, T = oracle.transmit(iface, phi_i, water, water, 0.0, "global")
    assert np.allclose(T, 1.0, atol=1e-15)
    tq = np.array([[0, 0, 15e-3], [2e-3, 1e-3, 25e-3], [-4e-3, 0, 40e-3]])
    got = oracle.rsi_field(iface, sigma, points(tq), k)
    want = oracle.piston_field(pist, points(tq), k)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-5


def test_density_step_scales_by_T():
    # same sound speed, different density: T12 = 2 rho1 / (rho1 + rho2) at every
    # angle and the transmitted field is T12 times the direct one.
    a, k, zi = 3e-3, 2 * np.pi / 2e-3, 10e-3
    pist = disk_quadrature(a, n_r=16, n_t=48)
    iface = plane_quadrature(0.04, 1.6e-3, 12, z0=zi, window=(0.016, 0.04))
    phi_i = oracle.piston_field(pist, iface, k)
    m1, m2 = {"rho": 1000.0, "c": 1480.0}, {"rho": 3000.0, "c": 1480.0}
    sigma, T = oracle.transmit(iface, phi_i, m1, m2, math.sin(0.2) / 1480.0, "global")
    assert np.allclose(T, 0.5, atol=1e-15)
    tq = np.array([[0, 0, 20e-3], [3e-3, 0, 30e-3]])
    got = oracle.rsi_field(iface, sigma, points(tq), k)
    want = 0.5 * oracle.piston_field(pist, points(tq), k)
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-5


def test_qmc_matched_impedance_chain():
    # the same invariant through the QMC point sets the workloads use
    water = {"rho": 1000.0, "c": 1480.0}
    cfg = {"freq": 2.0e6, "v0": 1.0, "seed": 0,
           "piston": {"a": 6.35e-3, "centre": (0, 0, 0), "tilt": 0.0, "n": 1 << 12, "set_id": 0},
           "media": [water, water],
           "interfaces": [{"kind": "rect", "centre": (0, 0, 0.02), "wx": 0.06, "wy": 0.06,
                           "n": 1 << 15, "set_id": 1}],
           "tmode": "global", "grid": {"x0": 0, "x1": 0, "nx": 1, "z0": 0, "z1": 0, "nz": 1}}
    tq = points([[0, 0, 0.04], [0, 0, 0.06], [2e-3, 0, 0.05]])
    got, _ = oracle.chain(cfg, tq)
    k = oracle.wavenumber(2.0e6, 1480.0)
    want = oracle.piston_field(disk_quadrature(6.35e-3), tq, k)
    assert rel(got, want) < 2e-2


def test_brute_force_tiny_inputs():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(3)
    src = {"x": rng.normal(size=3) * 1e-3, "y": rng.normal(size=3) * 1e-3,
           "z": rng.normal(size=3) * 1e-4, "nx": np.array([0.1, 0.0, -0.2]),
           "ny": np.array([0.0, 0.3, 0.1]), "nz": np.array([0.99, 0.95, 0.97]),
           "w": np.array([1e-6, 2e-6, 1.5e-6])}
    sigma = np.array([1 + 2j, -0.5 + 0.1j, 0.3 - 0.7j])
    tgt = points([[1e-3, 0, 5e-3], [0, -2e-3, 8e-3]])
    k = 2 * np.pi * 3e6 / 1480.0
    got_p = oracle.piston_field(src, tgt, k, 1.5)
    got_r = oracle.rsi_field(src, sigma, tgt, k)
    lam = 2 * mp.pi / mp.mpf(k)
    for j in range(2):
        accp, accr = mp.mpc(0), mp.mpc(0)
        for i in range(3):
            dx = mp.mpf(tgt["x"][j]) - mp.mpf(src["x"][i])
            dy = mp.mpf(tgt["y"][j]) - mp.mpf(src["y"][i])
            dz = mp.mpf(tgt["z"][j]) - mp.mpf(src["z"][i])
            r = mp.sqrt(dx * dx + dy * dy + dz * dz)
            e = mp.exp(1j * mp.mpf(k) * r) / r
            accp += -mp.mpf(1.5) / (2 * mp.pi) * mp.mpf(src["w"][i]) * e
            cth = (mp.mpf(src["nx"][i]) * dx + mp.mpf(src["ny"][i]) * dy
                   + mp.mpf(src["nz"][i]) * dz) / r
            s = mp.mpc(sigma[i].real, sigma[i].imag)
            accr += (-1j / lam) * mp.mpf(src["w"][i]) * s * e * (1 - 1 / (1j * mp.mpf(k) * r)) * cth
        # FP64 rounding of the phase k r (~60 rad here) bounds the agreement
        tol = 8 * k * 1e-2 * 2.0**-53 + 1e-15
        assert abs(complex(accp) - got_p[j]) <= tol * abs(complex(accp))
        assert abs(complex(accr) - got_r[j]) <= tol * abs(complex(accr))


def test_coincident_points_contribute_nothing():
    src = {"x": np.array([0.0, 1e-3]), "y": np.zeros(2), "z": np.zeros(2),
           "nx": np.zeros(2), "ny": np.zeros(2), "nz": np.ones(2), "w": np.ones(2)}
    tgt = points([[0.0, 0.0, 0.0]])
    k = 1000.0
    only_far = {key: v[1:] for key, v in src.items()}
    assert oracle.piston_field(src, tgt, k)[0] == oracle.piston_field(only_far, tgt, k)[0]
    sig = np.array([1.0 + 0j, 2.0 + 1j])
    assert oracle.rsi_field(src, sig, tgt, k)[0] == oracle.rsi_field(only_far, sig[1:], tgt, k)[0]


# ---------------------------------------------------------------------------
# interface coefficients (Eqs. reflection_coefficient, transmission_coefficient)
# ---------------------------------------------------------------------------
WATER = (1000.0, 1480.0)
STEEL = (7800.0, 5900.0)


def _cosines(c1, c2, a1):
    s2 = c2 / c1 * math.sin(a1)
    cos2 = math.sqrt(1 - s2 * s2) if s2 <= 1 else 1j * math.sqrt(s2 * s2 - 1)
    return math.cos(a1), cos2


@pytest.mark.parametrize("m1,m2", [(WATER, STEEL), (STEEL, WATER), ((1600.0, 3000.0), (1200.0, 2600.0))])
def test_T_identity_and_energy_balance(m1, m2):
    (r1, c1), (r2, c2) = m1, m2
    for deg in np.linspace(0.0, 80.0, 41):
        cos1, cos2 = _cosines(c1, c2, math.radians(deg))
        T = oracle.T12(r1, c1, r2, c2, cos1, cos2)
        R = oracle.R12(r1, c1, r2, c2, cos1, cos2)
        assert abs(r1 / r2 * (1 + R) - T) < 1e-14 * max(1.0, abs(T))
        if isinstance(cos2, complex):  # post-critical: total reflection
            assert abs(abs(R) - 1.0) < 1e-14
        else:  # normal energy flux conservation for the velocity potential
            p_t = r2 * T / r1  # pressure transmission ratio
            lhs = (1 - abs(R) ** 2) * cos1 / (r1 * c1)
            rhs = abs(p_t) ** 2 * cos2 / (r2 * c2)
            assert abs(lhs - rhs) < 1e-13 * max(lhs, 1e-300)


def test_transmit_modes_and_branch():
    pts = oracle.make_points({"kind": "rect", "centre": (0, 0, 0.05), "wx": 0.06, "wy": 0.06},
                             0, 1, 256)
    phi = np.exp(1j * np.arange(256) * 0.1)
    water, steel = {"rho": 1000.0, "c": 1480.0}, {"rho": 7800.0, "c": 5900.0}
    for deg in (0.0, 5.0, 14.0, 15.0, 30.0):
        C = math.sin(math.radians(deg)) / 1480.0
        sg, Tg = oracle.transmit(pts, phi, water, steel, C, "global")
        sl, Tl = oracle.transmit(pts, phi, water, steel, C, "local")
        # on a flat interface the local angle is the global one
        assert np.allclose(Tg, Tl, rtol=1e-13, atol=0)
        assert np.allclose(sg, Tg * phi, rtol=1e-15)
        crit = math.degrees(math.asin(1480.0 / 5900.0))
        if deg > crit:
            assert np.all(np.abs(Tg.imag) > 0)  # complex T after the critical angle
    # normal incidence, water -> steel
    _, T0 = oracle.transmit(pts, phi, water, steel, 0.0, "global")
    assert np.allclose(T0, 2 * 1000 * 5900 / (7800 * 5900 + 1000 * 1480))


def test_local_mode_on_cylinder_apex_matches_global():
    pts = oracle.make_points({"kind": "cyl", "centre": (0, 0, 0.03), "wx": 0.06, "wy": 0.06,
                              "R": 0.1}, 0, 2, 1024)
    water, lay = {"rho": 1000.0, "c": 1480.0}, {"rho": 1600.0, "c": 3000.0}
    _, Tl = oracle.transmit(pts, np.ones(1024), water, lay, 0.0, "local")
    _, Tg = oracle.transmit(pts, np.ones(1024), water, lay, 0.0, "global")
    cosl = pts["nz"]  # beam along +z: local incidence cosine is n_z
    near = np.abs(pts["x"]) < 1e-3
    assert np.allclose(Tl[near], Tg[near], rtol=1e-4)
    # the local coefficient is that of the plane-wave formula at the local angle
    for i in range(0, 1024, 97):
        c1 = cosl[i]
        s2 = 3000.0 / 1480.0 * math.sqrt(1 - c1 * c1)
        cos2 = math.sqrt(1 - s2 * s2) if s2 <= 1 else 1j * math.sqrt(s2 * s2 - 1)
        R = oracle.R12(1000.0, 1480.0, 1600.0, 3000.0, c1, cos2)
        assert abs(Tl[i] - 1000.0 / 1600.0 * (1 + R)) < 1e-14


def test_two_matched_interfaces_chain():
    # stage chaining (interface -> interface -> field) with identical media keeps
    # reproducing the direct field
    water = {"rho": 1000.0, "c": 1480.0}
    iface = lambda z, s: {"kind": "rect", "centre": (0, 0, z), "wx": 0.05, "wy": 0.05,
                          "n": 1 << 14, "set_id": s}
    cfg = {"freq": 1.5e6, "v0": 1.0, "seed": 0,
           "piston": {"a": 6.35e-3, "centre": (0, 0, 0), "tilt": 0.0, "n": 1 << 12, "set_id": 0},
           "media": [water, water, water],
           "interfaces": [iface(0.015, 1), iface(0.02, 2)],
           "tmode": "global", "grid": {"x0": 0, "x1": 0, "nx": 1, "z0": 0, "z1": 0, "nz": 1}}
    tq = points([[0, 0, 0.035], [0, 0, 0.05], [1e-3, 0, 0.045]])
    got, kept = oracle.chain(cfg, tq, keep=True)
    assert len(kept) == 2
    k = oracle.wavenumber(1.5e6, 1480.0)
    want = oracle.piston_field(disk_quadrature(6.35e-3), tq, k)
    assert rel(got, want) < 4e-2


def test_field_image_is_normalised_chain():
    water, steel = {"rho": 1000.0, "c": 1480.0}, {"rho": 7800.0, "c": 5900.0}
    cfg = {"freq": 3e6, "v0": 2.0, "seed": 1,
           "piston": {"a": 5e-3, "centre": (0, 0, 0), "tilt": 0.05, "n": 300, "set_id": 0},
           "media": [water, steel],
           "interfaces": [{"kind": "rect", "centre": (0, 0, 0.02), "wx": 0.03, "wy": 0.03,
                           "n": 500, "set_id": 1}],
           "tmode": "global",
           "grid": {"x0": -0.01, "x1": 0.01, "nx": 5, "z0": 0.02, "z1": 0.03, "nz": 3, "y": 0.0}}
    img = oracle.field_image(cfg)
    phi, _ = oracle.chain(cfg)
    assert img.shape == (3, 5)
    assert np.allclose(img.ravel(), oracle.wavenumber(3e6, 5900.0) / 2.0 * phi, rtol=1e-15)


# ---------------------------------------------------------------------------
# reflected field in medium 1 (Sec. 2.1, plane-wave reflection approximation)
# ---------------------------------------------------------------------------
def test_reflection_from_a_denser_plane_is_the_scaled_image_source():
    # Equal sound speeds, rho2 = 3 rho1: R12 = (rho2 - rho1)/(rho2 + rho1) = 1/2
    # at every angle.  A point source at z = -d below the plane z = 0 leaves
    # the reflected value R12 e^{ikR}/R on the plane; the first
    # Rayleigh-Sommerfeld solution with the normal pointing back into medium 1
    # reproduces the outgoing field of the mirror source at z = +d, times R12,
    # everywhere in z < 0.  Keeping the stored +z normal gives exactly the
    # negative, so the reversed normals are what this pins.
    k = 2 * np.pi / 1e-3
    d = 4e-3
    src = plane_quadrature(0.03, 0.75e-3, 12, window=(0.012, 0.03))
    R = np.sqrt(src["x"] ** 2 + src["y"] ** 2 + d * d)
    phi_i = np.exp(1j * k * R) / R
    m1, m2 = {"rho": 1000.0, "c": 1480.0}, {"rho": 3000.0, "c": 1480.0}
    sig_r, Rc = oracle.reflect(src, phi_i, m1, m2, math.sin(0.3) / 1480.0, "global")
    assert np.allclose(Rc, 0.5, atol=1e-15)
    tq = np.array([[0, 0, -5e-3], [3e-3, 2e-3, -10e-3], [0, 0, -0.4e-3], [1e-3, 0, -1.5e-3]])
    got = oracle.rsi_field(oracle.flip_normals(src), sig_r, points(tq), k)
    Rq = np.sqrt(tq[:, 0] ** 2 + tq[:, 1] ** 2 + (tq[:, 2] - d) ** 2)
    want = 0.5 * np.exp(1j * k * Rq) / Rq
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-6
    unflipped = oracle.rsi_field(src, sig_r, points(tq), k)
    assert np.allclose(unflipped, -got, rtol=1e-12, atol=0)


def test_reflection_coefficient_matches_its_closed_forms():
    # Normal incidence: R12 = (Z2 - Z1)/(Z2 + Z1); past the critical angle
    # |R12| = 1; and 1 + R12 = (rho2/rho1) T12 (Eq. reflection_coefficient
    # against Eq. transmission_coefficient), point by point.
    w, st = {"rho": 1000.0, "c": 1480.0}, {"rho": 7800.0, "c": 5900.0}
    pts = {"nx": np.zeros(3), "ny": np.zeros(3), "nz": np.ones(3)}
    phi = np.array([1.0, 2.0 - 1.0j, 0.5j])
    sig, R = oracle.reflect(pts, phi, w, st, 0.0, "global")
    z1, z2 = 1000.0 * 1480.0, 7800.0 * 5900.0
    assert np.allclose(R, (z2 - z1) / (z2 + z1), rtol=1e-15)
    assert np.allclose(sig, R * phi, rtol=1e-15)
    C = math.sin(math.radians(20.0)) / 1480.0  # beyond the first critical angle (14.5 deg)
    _, Rp = oracle.reflect(pts, phi, w, st, C, "global")
    assert np.allclose(np.abs(Rp), 1.0, rtol=1e-14)
    for C in (0.0, math.sin(math.radians(7.0)) / 1480.0, math.sin(math.radians(20.0)) / 1480.0):
        _, Rr = oracle.reflect(pts, phi, w, st, C, "global")
        _, T = oracle.transmit(pts, phi, w, st, C, "global")
        assert np.allclose(1.0 + Rr, (7800.0 / 1000.0) * T, rtol=1e-14)


def test_two_medium_matched_media_reflect_nothing():
    # Identical media: R12 = 0, so medium 1 holds the incident field alone and
    # medium 2 is the single-interface chain of the same points.
    from paper_2408_06765_gb300 import workloads as W
    cfg = W.f1_small()
    cfg["media"] = [dict(W.WATER), dict(W.WATER)]
    cfg["piston"]["n"], cfg["interfaces"][0]["n"] = 600, 900
    parts = oracle.two_medium(cfg, parts=True)
    assert np.all(parts["reflected"] == 0)
    img = oracle.two_medium(cfg)
    gw, gs = cfg["grid_water"], cfg["grid_solid"]
    k = oracle.wavenumber(cfg["freq"], 1480.0)
    pist = oracle.make_points(dict(cfg["piston"], kind="disk"), 0, 0, 600)
    direct = oracle.piston_field(pist, oracle.grid_points(gw), k)
    assert np.array_equal(img[: gw["nz"]], k * direct.reshape(gw["nz"], gw["nx"]))
    below, _ = oracle.chain(dict(cfg, grid=gs))
    assert np.array_equal(img[gw["nz"]:], k * below.reshape(gs["nz"], gs["nx"]))
