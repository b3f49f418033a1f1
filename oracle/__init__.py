"""FP64 CPU oracle for the QMC Rayleigh-Sommerfeld-integral (RSI) beam model.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_2408_06765_gb300``) and imports
nothing from it; both sides are fed the same plain-data workload description.

The arithmetic lives in ``rsi_oracle.c`` (plain C, double precision, direct
loops in source-index order with Neumaier compensation).  This module builds
it with gcc, calls it through ctypes and chains the stages exactly in the
order of Sec. 2.1 of the paper:

    piston  --Eq. incident_field-->  interface 1
    interface s  --T12 (Eq. transmission_coefficient)-->  source density
    source density  --Eq. rayleigh_sommerfeld (Eq. approximated_transmitted_field)-->
        interface s+1 ... or the field-image grid
    image = k phi / v0   (normalisation of Fig. oblique_incidence)

Parity pins for every function are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsi_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile rsi_oracle.c into oracle/_build/liboracle.so (gcc, -O2, IEEE)."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp = os.path.join(_BUILD, "machine.txt")
    same_host = os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()
    if (not force and same_host and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    with open(stamp, "w") as f:
        f.write(platform.machine())
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_mix64.restype = ctypes.c_uint64
            L.orc_mix64.argtypes = [ctypes.c_uint64]
            L.orc_scramble_key.restype = ctypes.c_uint64
            L.orc_scramble_key.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32]
            L.orc_owen.restype = ctypes.c_uint32
            L.orc_owen.argtypes = [ctypes.c_uint32, ctypes.c_uint64]
            L.orc_sobol.restype = None
            L.orc_sobol.argtypes = [ctypes.c_uint64, ctypes.c_uint32, _I64, _I64,
                                    ctypes.c_int, _U32, _U32]
            L.orc_halton.restype = None
            L.orc_halton.argtypes = [_I64, _I64, _U32, _U32]
            for name, extra in (("orc_map_disk", 6), ("orc_map_rect", 5), ("orc_map_cyl", 6),
                                ("orc_map_cap", 7)):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [_I64, ctypes.c_int, _U32, _U32] + [ctypes.c_double] * extra + [_D] * 7
            L.orc_grid_points.restype = None
            L.orc_grid_points.argtypes = [ctypes.c_double, ctypes.c_double, _I64,
                                          ctypes.c_double, ctypes.c_double, _I64,
                                          ctypes.c_double, _D, _D, _D]
            L.orc_piston_field.restype = None
            L.orc_piston_field.argtypes = [_I64, _D, _D, _D, _D, ctypes.c_double,
                                           ctypes.c_double, _I64, _D, _D, _D, _D, _D,
                                           ctypes.c_int]
            L.orc_rsi_field.restype = None
            L.orc_rsi_field.argtypes = [_I64, _D, _D, _D, _D, _D, _D, _D, _D, _D,
                                        ctypes.c_double, _I64, _D, _D, _D, _D, _D,
                                        ctypes.c_int]
            for name in ("orc_T12_ri", "orc_R12_ri"):
                f = getattr(L, name)
                f.restype = None
                f.argtypes = [ctypes.c_double] * 8 + [_D]
            L.orc_transmit.restype = None
            L.orc_transmit.argtypes = [_I64, ctypes.c_int] + [ctypes.c_double] * 5 + [_D] * 9
            L.orc_ray_path.restype = None
            L.orc_ray_path.argtypes = [ctypes.c_double] * 5 + [_D]
            L.orc_raytrace_field.restype = None
            L.orc_raytrace_field.argtypes = [_I64, _D, _D, _D, _D] + [ctypes.c_double] * 8 + \
                [_I64, _D, _D, _D, _D, _D, ctypes.c_int]
            L.orc_reflect.restype = None
            L.orc_reflect.argtypes = [_I64, ctypes.c_int] + [ctypes.c_double] * 5 + [_D] * 9
            _lib = L
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _p(a, ctype=_D):
    return a.ctypes.data_as(ctype)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# QMC points and geometry (Sec. 2.3)
# ---------------------------------------------------------------------------
def mix64(z: int) -> int:
    return int(lib().orc_mix64(ctypes.c_uint64(z & (2**64 - 1))))


def scramble_key(seed: int, set_id: int, dim: int) -> int:
    return int(lib().orc_scramble_key(seed, set_id, dim))


def owen(x: int, key: int) -> int:
    return int(lib().orc_owen(x, key))


def sobol(seed: int, set_id: int, n: int, first: int = 0, scrambled: bool = True):
    """32-bit integer Sobol coordinates (dims 1-2) of points first..first+n-1."""
    su = np.empty(n, np.uint32)
    sv = np.empty(n, np.uint32)
    lib().orc_sobol(seed, set_id, first, n, 1 if scrambled else 0, _p(su, _U32), _p(sv, _U32))
    return su, sv


def halton(n: int, first: int = 0):
    """Integer Halton coordinates of points first+1 .. first+n (bases 2, 3):
    the base-2 radical inverse as a 32-bit fraction, the base-3 one as a
    fraction of 3^20."""
    su = np.empty(n, np.uint32)
    sv = np.empty(n, np.uint32)
    lib().orc_halton(first, n, _p(su, _U32), _p(sv, _U32))
    return su, sv


SEQUENCES = {"sobol": 0, "halton": 1}


def map_points(surface: dict, su, sv) -> dict:
    """Map integer QMC coordinates onto a surface (Eqs. circle_sampling,
    square_sampling; cylinder and spherical-cap variants; optional Gaussian
    apodisation of the disk and cap).  Returns x, y, z, nx, ny, nz, w."""
    su = np.ascontiguousarray(su, np.uint32)
    sv = np.ascontiguousarray(sv, np.uint32)
    n = su.shape[0]
    out = {k: np.empty(n, np.float64) for k in ("x", "y", "z", "nx", "ny", "nz", "w")}
    ptrs = [_p(out[k]) for k in ("x", "y", "z", "nx", "ny", "nz", "w")]
    c = [float(v) for v in surface["centre"]]
    kind = surface["kind"]
    seq = SEQUENCES[surface.get("sequence", "sobol")]
    apod = float(surface.get("apod", 0.0))
    L = lib()
    if kind == "disk":
        L.orc_map_disk(n, seq, _p(su, _U32), _p(sv, _U32), *c, float(surface.get("tilt", 0.0)),
                       float(surface["a"]), apod, *ptrs)
    elif kind == "rect":
        L.orc_map_rect(n, seq, _p(su, _U32), _p(sv, _U32), *c, float(surface["wx"]),
                       float(surface["wy"]), *ptrs)
    elif kind == "cyl":
        L.orc_map_cyl(n, seq, _p(su, _U32), _p(sv, _U32), *c, float(surface["wx"]),
                      float(surface["wy"]), float(surface["R"]), *ptrs)
    elif kind == "cap":
        L.orc_map_cap(n, seq, _p(su, _U32), _p(sv, _U32), *c, float(surface.get("tilt", 0.0)),
                      float(surface["a"]), float(surface["R"]), apod, *ptrs)
    else:
        raise ValueError(f"unknown surface kind {kind!r}")
    return out


def make_points(surface: dict, seed: int, set_id: int, n: int, scrambled: bool = True) -> dict:
    """Points of a surface in index order: scrambled Sobol (seed, set_id) or,
    with surface["sequence"] == "halton", the Halton points 1..n."""
    if surface.get("sequence", "sobol") == "halton":
        su, sv = halton(n)
    else:
        su, sv = sobol(seed, set_id, n, 0, scrambled)
    pts = map_points(surface, su, sv)
    pts["su"], pts["sv"] = su, sv
    return pts


def grid_points(grid: dict) -> dict:
    nx, nz = int(grid["nx"]), int(grid["nz"])
    n = nx * nz
    x, y, z = (np.empty(n, np.float64) for _ in range(3))
    lib().orc_grid_points(float(grid["x0"]), float(grid["x1"]), nx, float(grid["z0"]),
                          float(grid["z1"]), nz, float(grid.get("y", 0.0)), _p(x), _p(y), _p(z))
    return {"x": x, "y": y, "z": z}


# ---------------------------------------------------------------------------
# Stage sums (Sec. 2.1)
# ---------------------------------------------------------------------------
def piston_field(src: dict, tgt: dict, k: float, v0: float = 1.0, nthreads: int | None = None):
    """Eq. incident_field over weighted source points; returns complex128."""
    sx, sy, sz, sw = (_f64(src[key]) for key in ("x", "y", "z", "w"))
    tx, ty, tz = (_f64(tgt[key]) for key in ("x", "y", "z"))
    nt = tx.shape[0]
    ore = np.empty(nt, np.float64)
    oim = np.empty(nt, np.float64)
    lib().orc_piston_field(sx.shape[0], _p(sx), _p(sy), _p(sz), _p(sw), float(v0), float(k),
                           nt, _p(tx), _p(ty), _p(tz), _p(ore), _p(oim),
                           nthreads or default_threads())
    return ore + 1j * oim


def rsi_field(src: dict, sigma, tgt: dict, k: float, nthreads: int | None = None):
    """Eq. rayleigh_sommerfeld with source density sigma; returns complex128."""
    sx, sy, sz, snx, sny, snz, sw = (_f64(src[key]) for key in ("x", "y", "z", "nx", "ny", "nz", "w"))
    sigma = np.ascontiguousarray(sigma, np.complex128)
    sre = _f64(sigma.real)
    sim = _f64(sigma.imag)
    tx, ty, tz = (_f64(tgt[key]) for key in ("x", "y", "z"))
    nt = tx.shape[0]
    ore = np.empty(nt, np.float64)
    oim = np.empty(nt, np.float64)
    lib().orc_rsi_field(sx.shape[0], _p(sx), _p(sy), _p(sz), _p(snx), _p(sny), _p(snz), _p(sw),
                        _p(sre), _p(sim), float(k), nt, _p(tx), _p(ty), _p(tz), _p(ore), _p(oim),
                        nthreads or default_threads())
    return ore + 1j * oim


def T12(rho1, c1, rho2, c2, cos1, cos2) -> complex:
    out = np.empty(2, np.float64)
    cos1, cos2 = complex(cos1), complex(cos2)
    lib().orc_T12_ri(rho1, c1, rho2, c2, cos1.real, cos1.imag, cos2.real, cos2.imag, _p(out))
    return complex(out[0], out[1])


def R12(rho1, c1, rho2, c2, cos1, cos2) -> complex:
    out = np.empty(2, np.float64)
    cos1, cos2 = complex(cos1), complex(cos2)
    lib().orc_R12_ri(rho1, c1, rho2, c2, cos1.real, cos1.imag, cos2.real, cos2.imag, _p(out))
    return complex(out[0], out[1])


TMODES = {"global": 0, "local": 1}


def transmit(pts: dict, phi, medium_in: dict, medium_out: dict, snell_C: float,
             mode: str = "global"):
    """Source density sigma = T12 phi on an interface; returns (sigma, T)."""
    nx, ny, nz = (_f64(pts[key]) for key in ("nx", "ny", "nz"))
    phi = np.ascontiguousarray(phi, np.complex128)
    pre, pim = _f64(phi.real), _f64(phi.imag)
    n = nx.shape[0]
    sre, sim, tre, tim = (np.empty(n, np.float64) for _ in range(4))
    lib().orc_transmit(n, TMODES[mode], float(medium_in["rho"]), float(medium_in["c"]),
                       float(medium_out["rho"]), float(medium_out["c"]), float(snell_C),
                       _p(nx), _p(ny), _p(nz), _p(pre), _p(pim), _p(sre), _p(sim),
                       _p(tre), _p(tim))
    return sre + 1j * sim, tre + 1j * tim


def reflect(pts: dict, phi, medium_in: dict, medium_out: dict, snell_C: float,
            mode: str = "global"):
    """Source density of the reflected field, sigma_r = R12 phi (the reflected
    field on the interface taken as R12 times the incident field, Sec. 2.1);
    returns (sigma_r, R)."""
    nx, ny, nz = (_f64(pts[key]) for key in ("nx", "ny", "nz"))
    phi = np.ascontiguousarray(phi, np.complex128)
    pre, pim = _f64(phi.real), _f64(phi.imag)
    n = nx.shape[0]
    sre, sim, rre, rim = (np.empty(n, np.float64) for _ in range(4))
    lib().orc_reflect(n, TMODES[mode], float(medium_in["rho"]), float(medium_in["c"]),
                      float(medium_out["rho"]), float(medium_out["c"]), float(snell_C),
                      _p(nx), _p(ny), _p(nz), _p(pre), _p(pim), _p(sre), _p(sim),
                      _p(rre), _p(rim))
    return sre + 1j * sim, rre + 1j * rim


def flip_normals(pts: dict) -> dict:
    """The same points with every normal reversed (pointing into the medium
    the field came from)."""
    return dict(pts, nx=-np.asarray(pts["nx"]), ny=-np.asarray(pts["ny"]), nz=-np.asarray(pts["nz"]))


# ---------------------------------------------------------------------------
# Whole chain: piston -> interfaces -> image (Sec. 2.1, Fig. rayleigh-sommerfeld_integral)
# ---------------------------------------------------------------------------
def wavenumber(freq: float, c: float) -> float:
    return 2.0 * math.pi * float(freq) / float(c)


def snell_invariant(cfg: dict) -> float:
    """C = sin(alpha)/c of the transducer axis in the first medium (Eq. root_searching)."""
    return math.sin(float(cfg["piston"].get("tilt", 0.0))) / float(cfg["media"][0]["c"])


def chain(cfg: dict, targets: dict | None = None, nthreads: int | None = None,
          keep: bool = False):
    """Run the stage chain of a workload description (see workloads module).

    Returns the field at `targets` (default: the image grid) and, with
    keep=True, the list of (points, phi-on-points) of every interface."""
    seed = int(cfg.get("seed", 0))
    freq = float(cfg["freq"])
    v0 = float(cfg.get("v0", 1.0))
    media = cfg["media"]
    C = snell_invariant(cfg)
    mode = cfg.get("tmode", "global")
    pc = cfg["piston"]
    piston = make_points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]))
    ifaces = []
    for it in cfg["interfaces"]:
        ifaces.append(make_points(it, seed, int(it["set_id"]), int(it["n"])))
    if targets is None:
        targets = grid_points(cfg["grid"])
    kept = []
    if not ifaces:
        return piston_field(piston, targets, wavenumber(freq, media[0]["c"]), v0, nthreads), kept
    phi = piston_field(piston, ifaces[0], wavenumber(freq, media[0]["c"]), v0, nthreads)
    for s, pts in enumerate(ifaces):
        if keep:
            kept.append((pts, phi))
        sigma, _ = transmit(pts, phi, media[s], media[s + 1], C, mode)
        nxt = ifaces[s + 1] if s + 1 < len(ifaces) else targets
        phi = rsi_field(pts, sigma, nxt, wavenumber(freq, media[s + 1]["c"]), nthreads)
    return phi, kept


def field_image(cfg: dict, nthreads: int | None = None):
    """Normalised image k phi / v0 on the workload's grid, shape [nz][nx]."""
    g = cfg["grid"]
    phi, _ = chain(cfg, None, nthreads)
    k_last = wavenumber(cfg["freq"], cfg["media"][len(cfg["interfaces"])]["c"])
    return (k_last / float(cfg.get("v0", 1.0))) * phi.reshape(int(g["nz"]), int(g["nx"]))


def two_medium(cfg: dict, nthreads: int | None = None, parts: bool = False, pixels=None):
    """Full field of a one-interface workload on both sides (Fig.
    rayleigh-sommerfeld_integral): in medium 1 the incident field (Eq.
    incident_field) plus the reflected field, the first Rayleigh-Sommerfeld
    solution over the interface with source density R12 phi_i, wave number
    k1 and normals pointing back into medium 1; in medium 2 the transmitted
    field (Eq. approximated_transmitted_field).  cfg["grid_water"] and
    cfg["grid_solid"] are the medium-1 and medium-2 windows (same nx).

    Returns the normalised image k phi / v0, shape [nz_w + nz_s][nx] (medium-1
    rows first), with `pixels` (flat indices into that image) only those
    values, or with parts=True a dict of its fields."""
    seed = int(cfg.get("seed", 0))
    freq, v0 = float(cfg["freq"]), float(cfg.get("v0", 1.0))
    m = cfg["media"]
    C = snell_invariant(cfg)
    mode = cfg.get("tmode", "global")
    k1, k2 = wavenumber(freq, m[0]["c"]), wavenumber(freq, m[1]["c"])
    pc, it = cfg["piston"], cfg["interfaces"][0]
    piston = make_points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]))
    iface = make_points(it, seed, int(it["set_id"]), int(it["n"]))
    gw, gs = grid_points(cfg["grid_water"]), grid_points(cfg["grid_solid"])
    n_w = int(cfg["grid_water"]["nx"]) * int(cfg["grid_water"]["nz"])
    if pixels is not None:
        pixels = np.asarray(pixels, np.int64)
        pw, ps = pixels[pixels < n_w], pixels[pixels >= n_w] - n_w
        gw = {key: gw[key][pw] for key in ("x", "y", "z")}
        gs = {key: gs[key][ps] for key in ("x", "y", "z")}
    phi_if = piston_field(piston, iface, k1, v0, nthreads)
    sig_t, _ = transmit(iface, phi_if, m[0], m[1], C, mode)
    sig_r, _ = reflect(iface, phi_if, m[0], m[1], C, mode)
    phi_inc = piston_field(piston, gw, k1, v0, nthreads)
    phi_ref = rsi_field(flip_normals(iface), sig_r, gw, k1, nthreads)
    phi_tr = rsi_field(iface, sig_t, gs, k2, nthreads)
    if parts:
        return {"interface": phi_if, "incident": phi_inc, "reflected": phi_ref, "transmitted": phi_tr}
    if pixels is not None:  # pixels are sorted: medium-1 values first
        return np.concatenate([(k1 / v0) * (phi_inc + phi_ref), (k2 / v0) * phi_tr])
    w, sg = cfg["grid_water"], cfg["grid_solid"]
    top = (k1 / v0) * (phi_inc + phi_ref).reshape(int(w["nz"]), int(w["nx"]))
    bot = (k2 / v0) * phi_tr.reshape(int(sg["nz"]), int(sg["nx"]))
    return np.concatenate([top, bot], axis=0)


# ---------------------------------------------------------------------------
# Ray-tracing model (Sec. 2.2)
# ---------------------------------------------------------------------------
def ray_path(h1: float, h2: float, rho: float, c1: float, c2: float) -> dict:
    """The refracted ray of Eq. ray_tracing: Snell's invariant C, path lengths
    D1, D2 and the cosines of the two angles."""
    out = np.empty(5, np.float64)
    lib().orc_ray_path(float(h1), float(h2), float(rho), float(c1), float(c2), _p(out))
    return {"C": out[0], "D1": out[1], "D2": out[2], "cos1": out[3], "cos2": out[4]}


def raytrace_field(src: dict, tgt: dict, m1: dict, m2: dict, z_interface: float, k1: float, k2: float,
                   v0: float = 1.0, nthreads: int | None = None):
    """Eq. transmitted_ray_tracing over weighted transducer points (z < z_I)
    onto targets in medium 2 (z > z_I); returns complex128."""
    sx, sy, sz, sw = (_f64(src[key]) for key in ("x", "y", "z", "w"))
    tx, ty, tz = (_f64(tgt[key]) for key in ("x", "y", "z"))
    nt = tx.shape[0]
    ore = np.empty(nt, np.float64)
    oim = np.empty(nt, np.float64)
    lib().orc_raytrace_field(sx.shape[0], _p(sx), _p(sy), _p(sz), _p(sw), float(v0), float(m1["rho"]),
                             float(m1["c"]), float(m2["rho"]), float(m2["c"]), float(z_interface), float(k1),
                             float(k2), nt, _p(tx), _p(ty), _p(tz), _p(ore), _p(oim),
                             nthreads or default_threads())
    return ore + 1j * oim


def raytrace_image(cfg: dict, nthreads: int | None = None, pixels=None):
    """Normalised image k2 phi_t / v0 of the ray-tracing model on a
    one-interface workload's grid (the interface plane is its centre's z),
    shape [nz][nx], or the values at flat pixel indices."""
    seed = int(cfg.get("seed", 0))
    freq, v0 = float(cfg["freq"]), float(cfg.get("v0", 1.0))
    m = cfg["media"]
    pc = cfg["piston"]
    piston = make_points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]))
    zI = float(cfg["interfaces"][0]["centre"][2])
    g = cfg["grid"]
    tg = grid_points(g)
    if pixels is not None:
        tg = {key: tg[key][np.asarray(pixels)] for key in ("x", "y", "z")}
    k1, k2 = wavenumber(freq, m[0]["c"]), wavenumber(freq, m[1]["c"])
    phi = raytrace_field(piston, tg, m[0], m[1], zI, k1, k2, v0, nthreads)
    val = (k2 / v0) * phi
    return val if pixels is not None else val.reshape(int(g["nz"]), int(g["nx"]))
