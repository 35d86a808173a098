"""Parity rule shared by the GPU tests, smoke and the benchmark's checks.

  - census bits, Hamming costs, arms: bit-exact;
  - aggregated cost (Eq. 2): |gpu - oracle| <= 1e-4 * oracle + 1e-6;
  - disparities (Eq. 3, both reference views): identical to the FP64
    oracle's decision, except at pixels whose FP64 best and second-best
    aggregated costs lie within that tolerance (near ties, where any finite
    precision may pick either); those excused pixels are counted and held
    at <= 0.1 % of each map;
  - consistency-checked map: identical to the check applied to the GPU's own
    two maps (integer work, bit-exact), and against the oracle's FP64 final
    map it may differ only where a near tie of the left map at p, or of the
    right map at the partner x - d of p, explains it; again <= 0.1 %.

The oracle can also take the Eq. 3 decision with an FP32 Eq. 1 and fixed
point aggregation (`quantized=True`); how many GPU pixels differ from that
decision is recorded beside the excused counts as a diagnostic, not gated.
Every check appends a line to REPORT, printed at the end of the pytest run.
"""
import numpy as np

REL = 1e-4
ABS = 1e-6
MAX_EXCUSED = 1e-3

# (what, excused pixels, pixels checked, pixels differing from the oracle's
# FP32 / fixed-point decision or None)
REPORT = []


def tol(best):
    return REL * np.asarray(best) + ABS


def near_ties(best, second):
    """Pixels whose FP64 best and second-best aggregated costs lie within the
    cost tolerance."""
    return (np.asarray(second) - np.asarray(best)) <= tol(best)


def _record(what, excused, total, qdiff):
    REPORT.append((what, int(excused), int(total), None if qdiff is None else int(qdiff)))


class Tally:
    """Excused pixels of several checks of one configuration (row bands
    sampled from the same maps): the 0.1 % cap holds for the total, since
    near ties cluster on flat surfaces and a single band can hold more than
    its share.  Pass it as `tally=` to the checks, then call close()."""

    def __init__(self, what: str):
        self.what, self.excused, self.total = what, 0, 0

    def add(self, n: int, total: int) -> None:
        self.excused += int(n)
        self.total += int(total)

    def close(self) -> int:
        frac = self.excused / self.total if self.total else 0.0
        _record(self.what + " (all sampled checks)", self.excused, self.total, None)
        assert frac <= MAX_EXCUSED, f"{self.what}: excused fraction {frac:.5f} > {MAX_EXCUSED}"
        return self.excused


def check_disparity(got, want, best, second, what="disparity", qwant=None, tally=None):
    """got: GPU map; want, best, second: the oracle's FP64 decision and its
    two smallest aggregated costs on the same pixels; qwant: the oracle's
    FP32 / fixed-point decision (diagnostic only) or None.  The excused
    fraction is capped here, or by `tally` over several checks.  Returns the
    number of excused pixels."""
    got = np.asarray(got)
    n = _near_ties(got, want, best, second, what, cap=tally is None)
    if tally is not None:
        tally.add(n, got.size)
    qd = None if qwant is None else int((got != np.asarray(qwant)).sum())
    _record(what, n, got.size, qd)
    return n


def _near_ties(got, want, best, second, what, cap=True):
    got = np.asarray(got)
    want = np.asarray(want)
    near = near_ties(best, second)
    diff = got != want
    bad = diff & ~near
    excused = diff & near
    if bad.any():
        ys, xs = np.nonzero(bad)
        raise AssertionError(f"{what}: {int(bad.sum())} pixels differ outside near ties, "
                             f"first at (y={ys[0]}, x={xs[0]}): got {got[ys[0], xs[0]]}, "
                             f"want {want[ys[0], xs[0]]}")
    frac = excused.mean() if excused.size else 0.0
    if cap:
        assert frac <= MAX_EXCUSED, f"{what}: excused fraction {frac:.5f} > {MAX_EXCUSED}"
    return int(excused.sum())


def final_excusable(got, ref):
    """Pixels of a consistency-checked map where a difference from the
    oracle's FP64 final map is explained by near ties: of the left map at p,
    or of the right map at the partner x - d for d the oracle's left
    disparity or the GPU's final one."""
    got = np.asarray(got)
    rows, W = got.shape
    nl = near_ties(ref.best_l, ref.second_l)
    nr = near_ties(ref.best_r, ref.second_r)
    ys, xs = np.mgrid[0:rows, 0:W]
    ok = nl.copy()
    for d in (np.asarray(ref.disp_l, np.int64), got.astype(np.int64)):
        xq = xs - d
        valid = (d >= 0) & (xq >= 0) & (xq < W)
        hit = np.zeros_like(ok)
        hit[valid] = nr[ys[valid], xq[valid]]
        ok |= hit
    return ok


def check_final(got, ref, what="final map", tally=None):
    """GPU consistency-checked map against the oracle's FP64 final map
    (ref: oracle.match(...) on the same rows): differences only where near
    ties explain them, at most 0.1 % of the map (or of `tally`'s total).
    Returns the number of excused pixels."""
    got = np.asarray(got)
    diff = got != np.asarray(ref.disp)
    bad = diff & ~final_excusable(got, ref)
    if bad.any():
        ys, xs = np.nonzero(bad)
        raise AssertionError(f"{what}: {int(bad.sum())} pixels differ without a near tie to explain them, "
                             f"first at (y={ys[0]}, x={xs[0]}): got {got[ys[0], xs[0]]}, "
                             f"want {ref.disp[ys[0], xs[0]]}")
    n = int(diff.sum())
    frac = n / diff.size if diff.size else 0.0
    if tally is None:
        assert frac <= MAX_EXCUSED, f"{what}: excused fraction {frac:.5f} > {MAX_EXCUSED}"
    else:
        tally.add(n, diff.size)
    qd = None if ref.qdisp is None else int((got != ref.qdisp).sum())
    _record(what, n, got.size, qd)
    return n


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


NOTES = []   # other figures the tests report (free text, one line each)


def note(line: str) -> None:
    NOTES.append(line)


def summary_lines():
    """One line per check: excused pixels and the FP32-decision diagnostic."""
    out = list(NOTES)
    for what, n, total, qd in REPORT:
        s = f"{what}: {n} of {total} pixels excused at near ties ({100.0 * n / max(total, 1):.4f} %)"
        if qd is not None:
            s += f"; {qd} differ from the oracle's FP32 / fixed-point decision"
        out.append(s)
    return out
