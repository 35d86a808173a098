"""Autotuner for the matcher's tile shapes, per pair shape.

Three tile parameters decide how the work of a pair meets the memory
hierarchy and the SMs (dco_params.d_chunk, h_chunk, v_chunk):

- the pass width (disparities aggregated per pass): narrow passes keep a
  pass's horizontal-sum slices in L2 and bound the workspace, wide passes
  run fewer, larger launches of the two aggregation kernels (measured on
  GB300: one pass of 64 disparities beats two of 32 at 640x480, one pass of
  256 beats eight of 32 at 1920x1080);
- the outputs per block of the first 1-D pass and of the second: shorter
  blocks give more, smaller blocks (a fuller last wave, more blocks per SM)
  at the price of reading the arm_l1 halo on both sides of every block once
  more.

The tuner times candidates on a pair of the shape with CUDA events, one
parameter at a time (the pass width with automatic blocks, then the first
pass's blocks, then the second's), keeps a change only when it is faster by
more than 1 %, and caches the winning Tile per (W, H, D, order, arm limit,
GPU name) in a JSON file, so later processes and the batch and serving paths
reuse it (dco_pair_desc and dco_stream_desc carry a pair's tile).
Candidates whose slices would exceed `max_slice_bytes` are not tried.  Only
timing and bookkeeping live here; the work runs in libdco_stereo.so.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Optional, Sequence

from .binding import Tile

_LOCK = threading.Lock()
MAX_SLICE_BYTES = 1 << 30   # both views' slices of one pass
H_MAX_LEN = 1024            # prefix positions one first-pass block holds
V_MAX_LEN = 512             # prefix positions one second-pass block holds
GAIN = 0.99                 # a candidate must be faster than this fraction of the best so far


def cache_path() -> str:
    base = os.environ.get("DCO_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "dco", "tiles.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db: dict) -> None:
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def key(W: int, H: int, D: int, gpu: str, order: int = 0, L1: int = 34) -> str:
    return f"{gpu}|{W}x{H}|D{D}|o{order}|L{L1}"


def candidates(W: int, H: int, D: int, max_slice_bytes: int = MAX_SLICE_BYTES) -> list[int]:
    """Pass widths to try: multiples of 32 up to D, and D itself, whose
    slices (4 bytes per pixel, disparity of the pass and view) fit the cap;
    the narrowest (32, or D below it) always."""
    c = {min(D, v) for v in range(32, D + 32, 32)} | {D}
    ok = sorted(v for v in c if 8 * W * H * v <= max_slice_bytes)
    return ok or [min(D, 32)]


def first_pass_candidates(n: int, L1: int = 34) -> list[int]:
    """Block lengths of the first 1-D pass over lines of n positions: 0
    (automatic: whole lines up to 1024, else 512) and lines cut into k
    near-equal blocks (multiples of 32, at least 64) whose prefix range with
    its halo fits one block."""
    out = [0]
    for k in range(1, 9):
        c = -(-n // k)
        c = -(-c // 32) * 32
        if c < 64 or c >= n or c + 2 * L1 > H_MAX_LEN or c in out:
            continue
        if n > H_MAX_LEN and c == 512:
            continue   # the automatic choice
        out.append(c)
    return out[:6]


def second_pass_candidates(n: int, L1: int = 34) -> list[int]:
    """Block lengths of the second 1-D pass over lines of n positions: 0
    (automatic) and lines cut into k balanced blocks of at least 32 whose
    prefix range with its halo fits one block (one value per block count)."""
    auto = 1 if n <= V_MAX_LEN else -(-n // (V_MAX_LEN - 2 * 40))
    out, counts = [0], {auto}
    for k in range(1, 9):
        c = -(-n // k)
        if c < 32 or (c < n or n > V_MAX_LEN) and c > V_MAX_LEN - 2 * L1:
            continue
        nb = -(-n // c)
        if nb in counts:
            continue
        counts.add(nb)
        out.append(c)
    return out[:6]


def lookup(W: int, H: int, D: int, gpu: str, order: int = 0, L1: int = 34) -> Optional[Tile]:
    with _LOCK:
        v = _load().get(key(W, H, D, gpu, order, L1))
    return Tile(*v["tile"]) if v and "tile" in v else None


def _time_call(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def _params(base, t: Tile):
    from .binding import Params
    p = Params.default(**{f: getattr(base, f) for f, _ in Params._fields_}) if base is not None else Params.default()
    p.d_chunk, p.h_chunk, p.v_chunk = t
    return p


def tune_tiles(stereo, left, right, D: int, params=None, reps: int = 5, use_cache: bool = True,
               max_slice_bytes: int = MAX_SLICE_BYTES) -> Tile:
    """Fastest tile for this pair's shape (timed on this pair, the other
    parameters taken from `params`); cached per shape and GPU."""
    import torch

    W, H = int(left.shape[1]), int(left.shape[0])
    order = int(params.agg_order) if params is not None else 0
    L1 = int(params.arm_l1) if params is not None else 34
    gpu = torch.cuda.get_device_name(left.device)
    if use_cache:
        hit = lookup(W, H, D, gpu, order, L1)
        if hit is not None:
            return hit
    out = torch.empty((H, W), dtype=torch.int16, device=left.device)
    times: dict[str, float] = {}

    def run(t: Tile) -> float:
        p = _params(params, t)
        ms = _time_call(lambda: stereo.match(left, right, D, p, out), reps)
        times[",".join(str(v) for v in t)] = ms
        return ms

    # one parameter at a time: pass width, then the first pass's blocks
    # (along rows for order 0, columns for order 1), then the second's
    n1, n2 = (W, H) if order == 0 else (H, W)
    best = Tile()
    best_ms = float("inf")
    for dc in candidates(W, H, D, max_slice_bytes):
        t = Tile(dc, 0, 0)
        ms = run(t)
        if ms < best_ms * GAIN or best_ms == float("inf"):
            best, best_ms = t, ms
    for hc in first_pass_candidates(n1, L1)[1:]:
        t = best._replace(h_chunk=hc)
        ms = run(t)
        if ms < best_ms * GAIN:
            best, best_ms = t, ms
    for vc in second_pass_candidates(n2, L1)[1:]:
        t = best._replace(v_chunk=vc)
        ms = run(t)
        if ms < best_ms * GAIN:
            best, best_ms = t, ms
    with _LOCK:
        db = _load()
        db[key(W, H, D, gpu, order, L1)] = {"tile": list(best), "ms": times}
        _store(db)
    return best


def tune_shape(stereo, W: int, H: int, D: int, device: int = 0, reps: int = 5, use_cache: bool = True,
               max_slice_bytes: int = MAX_SLICE_BYTES, params=None) -> Tile:
    """Fastest tile for pairs of shape (W, H, D), timed on a seeded synthetic
    plane scene of that shape when no cached answer exists."""
    import torch
    from . import scenes

    order = int(params.agg_order) if params is not None else 0
    L1 = int(params.arm_l1) if params is not None else 34
    gpu = torch.cuda.get_device_name(device)
    if use_cache:
        hit = lookup(W, H, D, gpu, order, L1)
        if hit is not None:
            return hit
    s = scenes.plane_scene(W, H, D, 6, seed=scenes.seed_for(7, W * 7 + H * 3 + D),
                           drange=(2, max(2, D - 2)), noise_sigma=2.0, texture="mixed")
    dev = torch.device(f"cuda:{device}")
    L = torch.from_numpy(s.left).to(dev)
    R = torch.from_numpy(s.right).to(dev)
    return tune_tiles(stereo, L, R, D, params=params, reps=reps, use_cache=False, max_slice_bytes=max_slice_bytes)


def tune_batch(stereo, shapes: Sequence[tuple[int, int, int]], device: int = 0, **kw) -> list[Tile]:
    """Per-pair tiles for a batch of (W, H, D) shapes (each distinct shape
    tuned once)."""
    won = {}
    for sh in shapes:
        sh = tuple(int(v) for v in sh)
        if sh not in won:
            won[sh] = tune_shape(stereo, *sh, device=device, **kw)
    return [won[tuple(int(v) for v in sh)] for sh in shapes]
