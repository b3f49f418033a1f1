"""Writes sincos_poly.cuh: polynomial sine and cosine of one full turn,
sin(2 pi s) = s P(s^2) (degree 11) and cos(2 pi s) = Q(s^2) (degree 12) for
s in [-1/2, 1/2], evaluated on the FP32 FMA pipe by the stage kernels for part
of their pairs (the MUFU pipe takes the rest).

The coefficients are near-minimax fits written here from the Taylor series'
structure: Lawson's iteratively reweighted least squares (C. L. Lawson, 1961)
on a dense grid in double precision, then rounded to float.  The error in
float arithmetic with fused multiply-adds is a few 1e-7 (tests/test_sincos_poly.py).

    python paper_2408_06765_gb300/csrc/gen_sincos_poly.py   # rewrites the header
"""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SIN_TERMS, COS_TERMS = 6, 7


def fit(odd: bool, terms: int) -> np.ndarray:
    s = np.linspace(-0.5, 0.5, 200001)
    u = s * s
    A = np.stack([(s if odd else np.ones_like(s)) * u ** k for k in range(terms)], 1)
    y = np.sin(2 * np.pi * s) if odd else np.cos(2 * np.pi * s)
    w = np.ones_like(s)
    for _ in range(60):
        c, *_ = np.linalg.lstsq(A * w[:, None], y * w, rcond=None)
        e = A @ c - y
        w = w * (np.abs(e) / np.abs(e).max() + 1e-3) ** 0.5
        w /= w.max()
    return c


def coefficients():
    return fit(True, SIN_TERMS).astype(np.float32), fit(False, COS_TERMS).astype(np.float32)


def header() -> str:
    sc, cc = coefficients()
    fmt = lambda v: f"{float(v):.9e}f"
    lines = [
        "// sincos_poly.cuh -- written by gen_sincos_poly.py (do not edit): sine and",
        "// cosine of a full turn on the FP32 FMA pipe, s in [-1/2, 1/2]:",
        "//   sin(2 pi s) = s (S0 + S1 u + ... + S5 u^5),  cos(2 pi s) = C0 + C1 u + ... + C6 u^6,  u = s^2",
        "// (near-minimax fits by Lawson's reweighted least squares, rounded to float).",
        "#pragma once",
        "",
    ]
    lines += [f"#define RSI_POLY_S{k} {fmt(v)}" for k, v in enumerate(sc)]
    lines += [f"#define RSI_POLY_C{k} {fmt(v)}" for k, v in enumerate(cc)]
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    with open(os.path.join(HERE, "sincos_poly.cuh"), "w") as f:
        f.write(header())
