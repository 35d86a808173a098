"""Python front end of the FP64 CPU oracle (ctypes over oracle/dco_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline / reference arm.  The product path never imports it.

Functions follow arXiv 2203.02300 Sect. 4:
  grey / census  -- census transform input (Sect. 4.2.1)
  arms           -- cross-support window (Sect. 4.1)
  cost_terms     -- Eq. 1 (AD-census robust combination, adaptive alpha)
  match          -- Eqs. 1-3 for both reference views + LR consistency
  lr_check       -- outlier removal by left-right consistency (Sect. 4.3 reading)
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i = ctypes.c_int
        d = ctypes.c_double
        L.orc_grey.argtypes = [P, i, i, P]
        L.orc_census.argtypes = [P, i, i, i, i, P]
        L.orc_hamming.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_arms.argtypes = [P, i, i, i, i, i, i, P]
        L.orc_alpha.argtypes = [i, d, d]
        L.orc_alpha.restype = d
        L.orc_cost_terms.argtypes = [i, i, i, d, d, d, d]
        L.orc_cost_terms.restype = d
        L.orc_lr_check.argtypes = [P, P, i, i, i, P]
        L.orc_match.argtypes = [P, P, i, i, i, i, d, d, d, d, i, i, i, i, i, i, i, i, i, i, i] + [P] * 11
        L.orc_arms_smooth.argtypes = [P, i, i, P]
        L.orc_arms_smooth.restype = i
        L.orc_vote.argtypes = [P, P, i, i, i, i, i, P]
        L.orc_vote.restype = i
        L.orc_downscale.argtypes = [P, i, i, P]
        L.orc_downscale.restype = i
        L.orc_depth.argtypes = [P, i, i, d, d, P]
        L.orc_depth.restype = i
        L.orc_grey.restype = i
        L.orc_census.restype = i
        L.orc_hamming.restype = i
        L.orc_arms.restype = i
        L.orc_lr_check.restype = i
        L.orc_match.restype = i
        _lib = L
    return _lib


@dataclasses.dataclass
class Params:
    """Matcher parameters: Sect. 7.2 values plus the readings for unstated ones."""
    lambda_ad: float = 10.0       # Sect. 7.2
    lambda_census: float = 40.0   # Sect. 7.2
    gamma_l: float = 1.0          # Sect. 7.2
    eps: float = 0.8              # Sect. 7.2
    census_w: int = 9             # reading (not stated)
    census_h: int = 7             # reading (not stated)
    arm_l1: int = 34              # reading (Sect. 4.1 cites the double threshold only)
    arm_l2: int = 17
    tau1: int = 20
    tau2: int = 6
    lr_tol: int = 1               # reading; < 0 disables the check
    smooth_arms: int = 0          # reading of Sect. 4.1's morphological processing; 1 = 3x3 opening
    agg_order: int = 0            # 0: region H then V (Eq. 2 reading); 1: V then H (variant)
    d_min: int = 0                # Eq. 3: d in [d_min, d_min + D - 1]


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int):
    if rc != 0:
        raise RuntimeError(f"oracle error code {rc}")


def _rgb(img: np.ndarray) -> np.ndarray:
    img = np.ascontiguousarray(img, dtype=np.uint8)
    assert img.ndim == 3 and img.shape[2] == 3
    return img


def grey(img: np.ndarray) -> np.ndarray:
    img = _rgb(img)
    H, W, _ = img.shape
    out = np.empty((H, W), np.int32)
    _check(lib().orc_grey(_ptr(img), W, H, _ptr(out)))
    return out


def census(img: np.ndarray, cw: int = 9, ch: int = 7) -> np.ndarray:
    img = _rgb(img)
    H, W, _ = img.shape
    out = np.empty((H, W), np.uint64)
    _check(lib().orc_census(_ptr(img), W, H, cw, ch, _ptr(out)))
    return out


def hamming(a: int, b: int) -> int:
    return int(lib().orc_hamming(ctypes.c_uint64(int(a)), ctypes.c_uint64(int(b))))


def arms(img: np.ndarray, p: Params = Params()) -> np.ndarray:
    """(H, W, 4) uint8 arm lengths {left, right, up, down}."""
    img = _rgb(img)
    H, W, _ = img.shape
    out = np.empty((H, W, 4), np.uint8)
    _check(lib().orc_arms(_ptr(img), W, H, p.arm_l1, p.arm_l2, p.tau1, p.tau2, _ptr(out)))
    if p.smooth_arms:
        _check(lib().orc_arms_smooth(_ptr(out), W, H, _ptr(out)))
    return out


def arms_smooth(arm: np.ndarray) -> np.ndarray:
    """Sect. 4.1 smoothing: grey-level 3x3 opening of each arm-length map."""
    arm = np.ascontiguousarray(arm, np.uint8)
    H, W, _ = arm.shape
    out = np.empty_like(arm)
    _check(lib().orc_arms_smooth(_ptr(arm), W, H, _ptr(out)))
    return out


def alpha(lmin: int, p: Params = Params()) -> float:
    return float(lib().orc_alpha(int(lmin), p.gamma_l, p.eps))


def cost_terms(ad_sum: int, ham: int, lmin: int, p: Params = Params()) -> float:
    return float(lib().orc_cost_terms(int(ad_sum), int(ham), int(lmin), p.lambda_ad,
                                      p.lambda_census, p.gamma_l, p.eps))


def lr_check(dl: np.ndarray, dr: np.ndarray, tol: int = 1) -> np.ndarray:
    dl = np.ascontiguousarray(dl, np.int16)
    dr = np.ascontiguousarray(dr, np.int16)
    rows, W = dl.shape
    out = np.empty_like(dl)
    _check(lib().orc_lr_check(_ptr(dl), _ptr(dr), W, rows, tol, _ptr(out)))
    return out


def vote(disp: np.ndarray, arm: np.ndarray, D: int, iters: int = 1, d_min: int = 0) -> np.ndarray:
    """Parallax optimisation (Sect. 4.3, Eq. 4): `iters` rounds of the mode of
    the valid disparities (those in [d_min, d_min + D - 1]) over each valid
    pixel's support region (arms of the reference view, (H, W, 4) uint8 l, r,
    u, d)."""
    disp = np.ascontiguousarray(disp, np.int16)
    arm = np.ascontiguousarray(arm, np.uint8)
    H, W = disp.shape
    assert arm.shape == (H, W, 4)
    out = np.empty_like(disp)
    _check(lib().orc_vote(_ptr(disp), _ptr(arm), W, H, D, d_min, iters, _ptr(out)))
    return out


def downscale(img: np.ndarray) -> np.ndarray:
    """Quarter-size input (Sect. 4): 2x2 rounded channel means, (H/2, W/2, 3)."""
    img = _rgb(img)
    H, W = img.shape[:2]
    out = np.empty((H // 2, W // 2, 3), np.uint8)
    _check(lib().orc_downscale(_ptr(img), W, H, _ptr(out)))
    return out


def depth(disp_half: np.ndarray, W: int, H: int, f: float, B: float) -> np.ndarray:
    """Sparse depth (Sect. 4.4): Z = f B / (2 d) on the 2x2 block of each
    half-size pixel of a W x H map; 0 where d <= 0."""
    disp_half = np.ascontiguousarray(disp_half, np.int16)
    assert disp_half.shape == (H // 2, W // 2)
    out = np.empty((H, W), np.float64)
    _check(lib().orc_depth(_ptr(disp_half), W, H, float(f), float(B), _ptr(out)))
    return out


@dataclasses.dataclass
class MatchResult:
    disp_l: np.ndarray     # (rows, W) int16, Eq. 3 on the left reference view
    disp_r: np.ndarray     # (rows, W) int16, Eq. 3 on the right reference view
    disp: np.ndarray       # (rows, W) int16, after the LR check (-1 invalid)
    best_l: np.ndarray     # (rows, W) float64 minimum aggregated cost (Eq. 2)
    second_l: np.ndarray   # (rows, W) float64 second-smallest aggregated cost
    best_r: np.ndarray
    second_r: np.ndarray
    vol_l: Optional[np.ndarray] = None   # (D, rows, W) aggregated costs, plane k for d = d_min + k
    vol_r: Optional[np.ndarray] = None
    y0: int = 0
    # Eq. 3 decisions taken in the kernel's precision (FP32 Eq. 1, fixed
    # point at scale S, exact integer region sums); None unless requested
    qdisp_l: Optional[np.ndarray] = None
    qdisp_r: Optional[np.ndarray] = None
    qdisp: Optional[np.ndarray] = None   # LR check of qdisp_l, qdisp_r


def match(left: np.ndarray, right: np.ndarray, D: int, p: Params = Params(),
          rows: Optional[tuple[int, int]] = None, volume: bool = False,
          quantized: bool = False) -> MatchResult:
    """Eqs. 1-3 for both reference views and the LR check on rows [y0, y1).
    quantized: also the Eq. 3 decisions in the kernel's precision (the paper
    fixes none; see the oracle's header for the recipe)."""
    left = _rgb(left)
    right = _rgb(right)
    H, W, _ = left.shape
    assert right.shape == left.shape
    y0, y1 = rows if rows is not None else (0, H)
    n = y1 - y0
    dl = np.empty((n, W), np.int16)
    dr = np.empty((n, W), np.int16)
    df = np.empty((n, W), np.int16)
    bl = np.empty((n, W)); sl = np.empty((n, W))
    br = np.empty((n, W)); sr = np.empty((n, W))
    vl = np.empty((D, n, W)) if volume else None
    vr = np.empty((D, n, W)) if volume else None
    ql = np.empty((n, W), np.int16) if quantized else None
    qr = np.empty((n, W), np.int16) if quantized else None
    null = ctypes.c_void_p(0)
    _check(lib().orc_match(_ptr(left), _ptr(right), W, H, D, p.d_min, p.lambda_ad, p.lambda_census,
                           p.gamma_l, p.eps, p.census_w, p.census_h, p.arm_l1, p.arm_l2,
                           p.tau1, p.tau2, p.lr_tol, p.smooth_arms, p.agg_order, y0, y1,
                           _ptr(dl), _ptr(dr), _ptr(df), _ptr(bl), _ptr(sl), _ptr(br), _ptr(sr),
                           _ptr(vl) if volume else null, _ptr(vr) if volume else null,
                           _ptr(ql) if quantized else null, _ptr(qr) if quantized else null))
    qf = lr_check(ql, qr, p.lr_tol) if quantized else None
    return MatchResult(dl, dr, df, bl, sl, br, sr, vl, vr, y0, ql, qr, qf)


def set_threads(n: int) -> None:
    """OpenMP thread count for subsequent oracle calls (0 = runtime default)."""
    if n > 0:
        os.environ["OMP_NUM_THREADS"] = str(n)
        try:
            gomp = ctypes.CDLL("libgomp.so.1")
            gomp.omp_set_num_threads(ctypes.c_int(n))
        except OSError:
            pass
