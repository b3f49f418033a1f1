"""Parity measure of the GPU tests: the relative L2 error over all values AND a
bound on the worst single value, max |got - want| <= 10 tol max |want|, so
that an error confined to a few pixels -- targets just below a source
surface, served by the kernels' near-pair path -- cannot hide in the norm of
a large image."""
import numpy as np

PIXEL_FACTOR = 10.0


def rel_l2(got, want) -> float:
    got, want = np.asarray(got).ravel(), np.asarray(want).ravel()
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def max_rel(got, want) -> float:
    """Worst absolute difference relative to the largest reference value."""
    got, want = np.asarray(got).ravel(), np.asarray(want).ravel()
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


def assert_close(got, want, tol: float, what: str = "") -> float:
    err, worst = rel_l2(got, want), max_rel(got, want)
    assert err <= tol, f"{what} relative L2 error {err:.3e} > {tol:.1e}"
    assert worst <= PIXEL_FACTOR * tol, (
        f"{what} worst value off by {worst:.3e} of the largest value > {PIXEL_FACTOR * tol:.1e}")
    return err
