"""Autotuner for the matcher's pass width (disparities aggregated per pass).

The pass width trades slice memory and L2 residency (narrow passes) against
fewer launches and less WTA-state traffic (wide passes).  The tuner times
each candidate on the caller's own inputs with CUDA events and caches the
winner per (W, H, D, GPU name) in a JSON file, so later processes reuse it.
Only timing and bookkeeping live here; the work runs in libdco_stereo.so.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Iterable, Optional

_LOCK = threading.Lock()


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


def candidates(D: int) -> list[int]:
    c = sorted({min(D, v) for v in (32, 64, 96, 128, 256)})
    return c


def lookup(W: int, H: int, D: int, gpu: str) -> Optional[int]:
    with _LOCK:
        v = _load().get(key(W, H, D, gpu))
    return int(v["d_chunk"]) if v else None


def tune_d_chunk(stereo, left, right, D: int, reps: int = 5,
                 cands: Optional[Iterable[int]] = None, use_cache: bool = True) -> int:
    """Fastest pass width for this pair's shape; cached per shape and GPU."""
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
    for dc in (cands or candidates(D)):
        p = Params.default(d_chunk=int(dc))
        stereo.match(left, right, D, p, out)
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            stereo.match(left, right, D, p, out)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        times[int(dc)] = best
    win = min(times, key=times.get)
    with _LOCK:
        db = _load()
        db[key(W, H, D, gpu)] = {"d_chunk": win, "ms": times}
        _store(db)
    return win
