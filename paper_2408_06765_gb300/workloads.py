"""Seeded synthetic workload descriptions for the RSI beam model.

This module holds inputs only -- geometry, media, point counts, seeds, image
grids -- as plain dictionaries.  It contains none of the method's arithmetic,
so both the CUDA path and the FP64 CPU oracle consume it.

Units are SI (m, s, kg/m^3, m/s, Hz).  Coordinates: z is depth (the beam
travels toward +z), the transducer face is centred at (x_t, 0, 0) and tilted
about +y, flat interfaces are planes z = z_I, field images are xz slices at
y = 0 stored row-major [nz][nx] with cell-centred pixels.

A description looks like::

    {"name": ..., "freq": Hz, "v0": 1.0, "seed": 0, "precision": "fp64"|"fp32c",
     "piston": {"a": m, "centre": (x, y, z), "tilt": rad, "n": N, "set_id": 0},
     "media": [{"rho": .., "c": ..}, ...],      # media[s] lies before interface s
     "interfaces": [{"kind": "rect"|"cyl", "centre": (..), "wx": m, "wy": m,
                     "R": m (cyl only), "n": N, "set_id": s}, ...],
     "tmode": "global"|"local",
     "grid": {"x0": m, "x1": m, "nx": .., "z0": m, "z1": m, "nz": .., "y": 0.0}}
"""
from __future__ import annotations

import math

import numpy as np

MM = 1e-3
MHZ = 1e6

WATER = {"rho": 1000.0, "c": 1480.0}
STEEL = {"rho": 7800.0, "c": 5900.0}  # longitudinal speed; shear speed is not used
LAYER_A = {"rho": 1600.0, "c": 3000.0}
LAYER_B = {"rho": 1200.0, "c": 2600.0}


def _rect(centre, w, n, set_id):
    return {"kind": "rect", "centre": tuple(centre), "wx": w, "wy": w, "n": int(n),
            "set_id": int(set_id)}


def c1_plain_fp64() -> dict:
    """Plain RSI in FP64: 6.35 mm piston, 5 MHz, water -> steel at z = 50 mm;
    4096 Sobol points on the piston and on a 60 x 60 mm patch; 64 x 64 image
    over a 40 x 40 mm window in the steel."""
    return {
        "name": "c1_plain_fp64", "freq": 5.0 * MHZ, "v0": 1.0, "seed": 0,
        "precision": "fp64",
        "piston": {"a": 6.35 * MM, "centre": (0.0, 0.0, 0.0), "tilt": 0.0, "n": 4096,
                   "set_id": 0},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((0.0, 0.0, 50 * MM), 60 * MM, 4096, 1)],
        "tmode": "global",
        "grid": {"x0": -20 * MM, "x1": 20 * MM, "nx": 64, "z0": 50 * MM, "z1": 90 * MM,
                 "nz": 64, "y": 0.0},
    }


C2_FREQS = (2.25 * MHZ, 5.0 * MHZ, 10.0 * MHZ)


def c2_full_image(freq: float) -> dict:
    """Full-image RSI, FP32 with a double-float phase: 2^16 piston points,
    2^18 points on an 80 x 80 mm patch, 512 x 512 image 60 mm deep."""
    return {
        "name": f"c2_full_image_{freq / MHZ:g}MHz", "freq": float(freq), "v0": 1.0,
        "seed": 0, "precision": "fp32c",
        "piston": {"a": 6.35 * MM, "centre": (0.0, 0.0, 0.0), "tilt": 0.0, "n": 1 << 16,
                   "set_id": 0},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((0.0, 0.0, 50 * MM), 80 * MM, 1 << 18, 1)],
        "tmode": "global",
        "grid": {"x0": -40 * MM, "x1": 40 * MM, "nx": 512, "z0": 50 * MM, "z1": 110 * MM,
                 "nz": 512, "y": 0.0},
    }


def c2_all() -> list[dict]:
    return [c2_full_image(f) for f in C2_FREQS]


def f1_two_medium(freq: float = 5.0 * MHZ, tilt_deg: float = 10.0, n_piston: int = 1 << 16,
                  n_iface: int = 1 << 18, nx: int = 512, nz_water: int = 256, nz_solid: int = 256,
                  half_width: float = 40 * MM, depth: float = 30 * MM, patch: float = 80 * MM) -> dict:
    """Both sides of c2's interface: the 6.35 mm piston tilted by 10 degrees,
    water -> steel at z = 50 mm, 2^16 piston points and 2^18 points on an
    80 x 80 mm patch centred where the axis meets the interface; the image
    (512 wide, 60 mm deep) holds the incident + reflected field in the 30 mm
    of water above the interface and the transmitted field in the 30 mm of
    steel below it."""
    tilt = math.radians(tilt_deg)
    zi = 50 * MM
    xc = zi * math.tan(tilt)
    return {
        "name": f"f1_two_medium_{freq / MHZ:g}MHz", "freq": float(freq), "v0": 1.0,
        "seed": 0, "precision": "fp32c",
        "piston": {"a": 6.35 * MM, "centre": (0.0, 0.0, 0.0), "tilt": tilt, "n": int(n_piston),
                   "set_id": 0},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((xc, 0.0, zi), patch, n_iface, 1)],
        "tmode": "global",
        "grid_water": {"x0": -half_width, "x1": half_width, "nx": int(nx), "z0": zi - depth, "z1": zi,
                       "nz": int(nz_water), "y": 0.0},
        "grid_solid": {"x0": -half_width, "x1": half_width, "nx": int(nx), "z0": zi, "z1": zi + depth,
                       "nz": int(nz_solid), "y": 0.0},
    }


def f2_ray_tracing(freq: float = 5.0 * MHZ, tilt_deg: float = 10.0, n_piston: int = 1 << 16,
                   nx: int = 512, nz: int = 512) -> dict:
    """The ray-tracing model (Sec. 2.2) on c2's geometry: the 6.35 mm piston
    tilted by 10 degrees with 2^16 points, water -> steel at z = 50 mm, a
    512 x 512 image over x in [-40, 40] mm, z in (50, 110] mm in the steel."""
    tilt = math.radians(tilt_deg)
    zi = 50 * MM
    return {
        "name": f"f2_ray_tracing_{freq / MHZ:g}MHz", "freq": float(freq), "v0": 1.0, "seed": 0,
        "piston": {"a": 6.35 * MM, "centre": (0.0, 0.0, 0.0), "tilt": tilt, "n": int(n_piston), "set_id": 0},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((zi * math.tan(tilt), 0.0, zi), 80 * MM, 0, 1)],  # the plane z = 50 mm
        "grid": {"x0": -40 * MM, "x1": 40 * MM, "nx": int(nx), "z0": zi, "z1": zi + 60 * MM, "nz": int(nz),
                 "y": 0.0},
    }


def f2_small() -> dict:
    """f2 at sizes the oracle finishes in a second: 3001 piston points (ragged
    tiles) onto 37 x 29 pixels reaching out to 75 degrees in the steel."""
    cfg = f2_ray_tracing(n_piston=3001, nx=37, nz=29)
    cfg["grid"].update({"x0": -30 * MM, "x1": 30 * MM, "z1": 50 * MM + 20 * MM})
    return cfg


def f3_halton(apod: float = 0.0) -> dict:
    """c1 with the paper's own point sets: Halton points 1..4096 on the
    piston and on the 60 x 60 mm patch (Sec. 2.3), FP32C; apod > 0 gives the
    piston a Gaussian velocity profile of that radius (Sec. 4)."""
    cfg = c1_plain_fp64()
    cfg["name"] = "f3_halton" + ("_apodised" if apod else "")
    cfg["precision"] = "fp32c"
    cfg["piston"].update({"sequence": "halton", "apod": float(apod)})
    cfg["interfaces"][0]["sequence"] = "halton"
    return cfg


F4_R = 33 * MM  # radius of curvature: focal length 14 mm in steel behind 10 mm of water (Sec. 3.3)


def f4_focused(freq: float = 2.5 * MHZ, n_piston: int = 1 << 16, n_iface: int = 1 << 18, nx: int = 512,
               nz: int = 512, patch: float = 40 * MM, half_width: float = 10 * MM, depth: float = 30 * MM) -> dict:
    """Focused transducer (Sec. 3.3, Fig. transducer_system b): a spherical
    cap of aperture radius 6.35 mm and radius of curvature 33 mm, 10 mm of
    water to the steel, 2.5 MHz; 2^16 points on the cap, 2^18 on a 40 x 40 mm
    patch (about three transducer diameters, Eq. square_sampling), 512 x 512
    image over x in [-10, 10] mm, z in (10, 40] mm of steel around the focus."""
    zi = 10 * MM
    return {
        "name": f"f4_focused_{freq / MHZ:g}MHz", "freq": float(freq), "v0": 1.0, "seed": 0, "precision": "fp32c",
        "piston": {"kind": "cap", "a": 6.35 * MM, "R": F4_R, "centre": (0.0, 0.0, 0.0), "tilt": 0.0,
                   "n": int(n_piston), "set_id": 0},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((0.0, 0.0, zi), patch, n_iface, 1)],
        "tmode": "global",
        "grid": {"x0": -half_width, "x1": half_width, "nx": int(nx), "z0": zi, "z1": zi + depth, "nz": int(nz),
                 "y": 0.0},
    }


def f4_small() -> dict:
    """f4 at sizes the oracle finishes in a second (ragged counts)."""
    return f4_focused(n_piston=3001, n_iface=6000, nx=37, nz=29, patch=20 * MM, half_width=5 * MM,
                      depth=15 * MM)


def f1_small() -> dict:
    """f1 at sizes the oracle finishes in a second, still resolving the
    water wavelength on the interface (2.25 MHz, 12 000 points on 40 mm):
    ragged point counts and an image of 48 x (20 + 24) pixels."""
    return f1_two_medium(freq=2.25 * MHZ, n_piston=3000, n_iface=12000, nx=48, nz_water=20, nz_solid=24,
                         half_width=15 * MM, depth=10 * MM, patch=40 * MM)


C3_TOP = 30 * MM
C3_LAYER = 0.5 * MM
C3_NLAYERS = 8
C3_R = 100 * MM


def c3_multilayer(curved: bool = False, n_per_surface: int = 1 << 16) -> dict:
    """Multilayer RSI: 5 mm piston, 5 MHz, 30 mm water path, 8 layers of
    0.5 mm alternating (3000 m/s, 1600) / (2600 m/s, 1200), water below,
    2^16 points per surface on 60 x 60 mm, 256 x 256 image below the stack.
    The curved variant makes the laminate concentric cylinders (axis parallel
    to y at depth 30 mm + 100 mm, top radius 100 mm) and uses the local
    incidence angle; its image window starts 4 mm deeper so that it clears
    the curved bottom surface."""
    media = [dict(WATER)]
    for i in range(C3_NLAYERS):
        media.append(dict(LAYER_A if i % 2 == 0 else LAYER_B))
    media.append(dict(WATER))
    ifaces = []
    for s in range(C3_NLAYERS + 1):
        zs = C3_TOP + s * C3_LAYER
        if curved:
            ifaces.append({"kind": "cyl", "centre": (0.0, 0.0, zs), "wx": 60 * MM,
                           "wy": 60 * MM, "R": C3_R - (zs - C3_TOP), "n": n_per_surface,
                           "set_id": s + 1})
        else:
            ifaces.append(_rect((0.0, 0.0, zs), 60 * MM, n_per_surface, s + 1))
    z_bot = C3_TOP + C3_NLAYERS * C3_LAYER
    z0 = z_bot + (4 * MM if curved else 0.0)
    return {
        "name": "c3_multilayer_curved" if curved else "c3_multilayer_flat",
        "freq": 5.0 * MHZ, "v0": 1.0, "seed": 0, "precision": "fp32c",
        "piston": {"a": 5.0 * MM, "centre": (0.0, 0.0, 0.0), "tilt": 0.0,
                   "n": n_per_surface, "set_id": 0},
        "media": media, "interfaces": ifaces,
        "tmode": "local" if curved else "global",
        "grid": {"x0": -20 * MM, "x1": 20 * MM, "nx": 256, "z0": z0, "z1": z0 + 40 * MM,
                 "nz": 256, "y": 0.0},
    }


C4_NFREQ = 64
C4_NPOS = 32


def c4_counts(seed: int = 0, n_instances: int = C4_NFREQ * C4_NPOS):
    """Per-instance QMC counts N = round(2^(12 + 4U)), U uniform from the
    counter-based Philox generator: columns (piston, interface)."""
    gen = np.random.Generator(np.random.Philox(key=seed))
    u = gen.random((n_instances, 2))
    return np.rint(np.exp2(12.0 + 4.0 * u)).astype(np.int64)


def c4_instance(j_freq: int, p_pos: int, counts) -> dict:
    """One instance of the broadband scan: f = 1 + 9 j/63 MHz, transducer at
    x = (p - 15.5) mm over the water -> steel interface of c1, 128 x 128 image
    over the c1 window."""
    inst = j_freq * C4_NPOS + p_pos
    x_t = (p_pos - 15.5) * MM
    n_p, n_i = (int(v) for v in counts[inst])
    return {
        "name": f"c4_f{j_freq}_p{p_pos}", "freq": (1.0 + 9.0 * j_freq / 63.0) * MHZ,
        "v0": 1.0, "seed": 0, "precision": "fp32c",
        "piston": {"a": 6.35 * MM, "centre": (x_t, 0.0, 0.0), "tilt": 0.0, "n": n_p,
                   "set_id": 2 * inst},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((x_t, 0.0, 50 * MM), 60 * MM, n_i, 2 * inst + 1)],
        "tmode": "global",
        "grid": {"x0": -20 * MM, "x1": 20 * MM, "nx": 128, "z0": 50 * MM, "z1": 90 * MM,
                 "nz": 128, "y": 0.0},
    }


def c4_all(seed: int = 0) -> list[dict]:
    counts = c4_counts(seed)
    return [c4_instance(j, p, counts) for j in range(C4_NFREQ) for p in range(C4_NPOS)]


def c5_params(n: int, seed: int = 0):
    """Surrogate inputs, uniform: x-offset [-10, 10] mm, tilt [-15, 15] deg,
    water path [20, 60] mm, frequency [2, 10] MHz, image depth below the
    interface [1, 20] mm.  Columns in SI units (tilt in radians)."""
    gen = np.random.Generator(np.random.Philox(key=seed + 0x5EED))
    u = gen.random((n, 5))
    lo = np.array([-10 * MM, math.radians(-15.0), 20 * MM, 2.0 * MHZ, 1 * MM])
    hi = np.array([10 * MM, math.radians(15.0), 60 * MM, 10.0 * MHZ, 20 * MM])
    return lo + (hi - lo) * u


def c5_instance(params, index: int = 0, n_piston: int = 1 << 14,
                n_iface: int = 1 << 16, n_img: int = 128) -> dict:
    """One surrogate training field: the water path is measured along the
    transducer axis, the interface patch (60 x 60 mm) is centred where the
    axis meets the interface, and the 40 x 40 mm image window is centred
    laterally on that point with its top edge `depth` below the interface."""
    x_off, tilt, path, freq, depth = (float(v) for v in params)
    z_i = path * math.cos(tilt)
    x_hit = x_off + path * math.sin(tilt)
    return {
        "name": f"c5_{index}", "freq": freq, "v0": 1.0, "seed": 0, "precision": "fp32c",
        "piston": {"a": 6.35 * MM, "centre": (x_off, 0.0, 0.0), "tilt": tilt,
                   "n": n_piston, "set_id": 2 * index},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((x_hit, 0.0, z_i), 60 * MM, n_iface, 2 * index + 1)],
        "tmode": "global",
        "grid": {"x0": x_hit - 20 * MM, "x1": x_hit + 20 * MM, "nx": n_img,
                 "z0": z_i + depth, "z1": z_i + depth + 40 * MM, "nz": n_img, "y": 0.0},
    }


def small_ragged(precision: str = "fp32c", freq: float = 5.0 * MHZ, tilt: float = 0.0,
                 n_piston: int = 1000, n_iface: int = 3000, nx: int = 37, nz: int = 29) -> dict:
    """A small case with counts that are not multiples of any tile size, for
    parity tests the oracle finishes in seconds."""
    return {
        "name": "small_ragged", "freq": freq, "v0": 1.0, "seed": 7, "precision": precision,
        "piston": {"a": 6.35 * MM, "centre": (1.0 * MM, 0.0, 0.0), "tilt": tilt,
                   "n": n_piston, "set_id": 0},
        "media": [dict(WATER), dict(STEEL)],
        "interfaces": [_rect((1.0 * MM, 0.0, 30 * MM), 40 * MM, n_iface, 1)],
        "tmode": "global",
        "grid": {"x0": -15 * MM, "x1": 17 * MM, "nx": nx, "z0": 30 * MM, "z1": 55 * MM,
                 "nz": nz, "y": 0.0},
    }


def pairs_of(cfg: dict) -> int:
    """Source x target pair count of one chain (piston stage + interface stages)."""
    n = [int(cfg["piston"]["n"])] + [int(it["n"]) for it in cfg["interfaces"]]
    n.append(int(cfg["grid"]["nx"]) * int(cfg["grid"]["nz"]))
    return sum(n[i] * n[i + 1] for i in range(len(n) - 1))
