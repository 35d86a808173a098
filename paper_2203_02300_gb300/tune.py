"""Autotuner for the matcher's pass width, per pair shape.

The pass width (disparities aggregated per pass, `d_chunk`) is the tile
parameter that decides how the cost slices meet the memory hierarchy: narrow
passes keep a pass's horizontal-sum slices in L2 and bound the workspace,
wide passes run fewer, larger launches of the horizontal and vertical
kernels.  Which wins depends on the pair's W x H x D (measured on GB300: one
pass of 64 disparities beats two of 32 at 640x480, one pass of 256 beats
eight of 32 at 1920x1080).  The tuner times each candidate on a pair of the
shape with CUDA events and caches the winner per (W, H, D, GPU name) in a
JSON file, so later processes and the batch and serving paths reuse it
(dco_pair_desc.d_chunk carries a pair's width into a batch).  Candidates
whose slices would exceed `max_slice_bytes` are not tried (the volume of
horizontal sums is only materialised as far as the memory allows).  Only
timing and bookkeeping live here; the work runs in libdco_stereo.so.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Iterable, Optional, Sequence

_LOCK = threading.Lock()
MAX_SLICE_BYTES = 1 << 30   # both views' slices of one pass


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


def key(W: int, H: int, D: int, gpu: str) -> str:
    return f"{gpu}|{W}x{H}|D{D}"


def candidates(W: int, H: int, D: int, max_slice_bytes: int = MAX_SLICE_BYTES) -> list[int]:
    """Pass widths to try: multiples of 32 up to D, and D itself, whose
    slices (4 bytes per pixel, disparity of the pass and view) fit the cap;
    the narrowest (32, or D below it) always."""
    c = {min(D, v) for v in range(32, D + 32, 32)} | {D}
    ok = sorted(v for v in c if 8 * W * H * v <= max_slice_bytes)
    return ok or [min(D, 32)]


def lookup(W: int, H: int, D: int, gpu: str) -> Optional[int]:
    with _LOCK:
        v = _load().get(key(W, H, D, gpu))
    return int(v["d_chunk"]) if v else None


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


def tune_d_chunk(stereo, left, right, D: int, reps: int = 5,
                 cands: Optional[Iterable[int]] = None, use_cache: bool = True,
                 max_slice_bytes: int = MAX_SLICE_BYTES) -> int:
    """Fastest pass width for this pair's shape (timed on this pair); cached
    per shape and GPU."""
    import torch
    from .binding import Params

    W, H = int(left.shape[1]), int(left.shape[0])
    gpu = torch.cuda.get_device_name(left.device)
    if use_cache:
        hit = lookup(W, H, D, gpu)
        if hit is not None:
            return hit
    out = torch.empty((H, W), dtype=torch.int16, device=left.device)
    times = {}
    for dc in (cands or candidates(W, H, D, max_slice_bytes)):
        p = Params.default(d_chunk=int(dc))
        times[int(dc)] = _time_call(lambda: stereo.match(left, right, D, p, out), reps)
    win = min(times, key=times.get)
    with _LOCK:
        db = _load()
        db[key(W, H, D, gpu)] = {"d_chunk": win, "ms": times}
        _store(db)
    return win


def tune_shape(stereo, W: int, H: int, D: int, device: int = 0, reps: int = 5, use_cache: bool = True,
               max_slice_bytes: int = MAX_SLICE_BYTES) -> int:
    """Fastest pass width for pairs of shape (W, H, D), timed on a seeded
    synthetic plane scene of that shape when no cached answer exists."""
    import torch
    from . import scenes

    gpu = torch.cuda.get_device_name(device)
    if use_cache:
        hit = lookup(W, H, D, gpu)
        if hit is not None:
            return hit
    s = scenes.plane_scene(W, H, D, 6, seed=scenes.seed_for(7, W * 7 + H * 3 + D),
                           drange=(2, max(2, D - 2)), noise_sigma=2.0, texture="mixed")
    dev = torch.device(f"cuda:{device}")
    L = torch.from_numpy(s.left).to(dev)
    R = torch.from_numpy(s.right).to(dev)
    return tune_d_chunk(stereo, L, R, D, reps=reps, use_cache=False, max_slice_bytes=max_slice_bytes)


def tune_batch(stereo, shapes: Sequence[tuple[int, int, int]], device: int = 0, **kw) -> list[int]:
    """Per-pair pass widths for a batch of (W, H, D) shapes (each distinct
    shape tuned once)."""
    won = {}
    for sh in shapes:
        sh = tuple(int(v) for v in sh)
        if sh not in won:
            won[sh] = tune_shape(stereo, *sh, device=device, **kw)
    return [won[tuple(int(v) for v in sh)] for sh in shapes]
