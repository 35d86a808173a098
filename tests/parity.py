"""Parity rule shared by the GPU tests, smoke and the benchmark's checks.

  - census bits, Hamming costs, arms: bit-exact;
  - aggregated cost (Eq. 2): |gpu - oracle| <= 1e-4 * oracle + 1e-6;
  - disparities (Eq. 3, both reference views): identical, except at pixels
    where the oracle's best and second-best aggregated costs lie within that
    tolerance (a near tie that rounding may break either way); such excused
    pixels must be <= 0.1 % of the map;
  - consistency map: identical to the consistency check applied to the GPU's
    own two disparity maps (integer work, bit-exact).
"""
import numpy as np

REL = 1e-4
ABS = 1e-6
MAX_EXCUSED = 1e-3


def tol(best):
    return REL * np.asarray(best) + ABS


def check_disparity(got, want, best, second, what="disparity"):
    got = np.asarray(got)
    want = np.asarray(want)
    near = (np.asarray(second) - np.asarray(best)) <= tol(best)
    diff = got != want
    bad = diff & ~near
    excused = diff & near
    if bad.any():
        ys, xs = np.nonzero(bad)
        raise AssertionError(f"{what}: {int(bad.sum())} pixels differ outside near ties, "
                             f"first at (y={ys[0]}, x={xs[0]}): got {got[ys[0], xs[0]]}, "
                             f"want {want[ys[0], xs[0]]}")
    frac = excused.mean() if excused.size else 0.0
    assert frac <= MAX_EXCUSED, f"{what}: excused fraction {frac:.5f} > {MAX_EXCUSED}"
    return int(excused.sum())


def check_cost(got, best, disp_got, disp_want, what="cost"):
    """GPU minimum aggregated cost against the oracle's minimum: within the
    tolerance where the disparities agree, within twice it at excused ties."""
    got = np.asarray(got, np.float64)
    best = np.asarray(best)
    t = np.where(np.asarray(disp_got) == np.asarray(disp_want), tol(best), 2 * tol(best))
    err = np.abs(got - best)
    if (err > t).any():
        i = np.unravel_index(np.argmax(err - t), err.shape)
        raise AssertionError(f"{what}: max excess at {i}: got {got[i]!r}, want {best[i]!r}")


def check_volume(got, want, what="volume"):
    got = np.asarray(got, np.float64)
    want = np.asarray(want)
    err = np.abs(got - want)
    t = tol(want)
    if (err > t).any():
        i = np.unravel_index(np.argmax(err - t), err.shape)
        raise AssertionError(f"{what}: element {i}: got {got[i]!r}, want {want[i]!r}")
    return float((err / np.maximum(want, 1e-30)).max())
