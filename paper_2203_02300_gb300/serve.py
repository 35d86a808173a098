"""Multi-stream serving loop with continuous batching (config 4).

Several camera streams, each with its own frame size and disparity range,
submit frames at their own rates.  The server keeps every stream's device
buffers resident (a few input/output slots per stream), and runs a
continuous-batching loop:

  - a frame is admitted into the next batch when its stream has a free slot
    and the batch's workspace (``dco_stereo_workspace_bytes`` summed over its
    pairs) still fits the lane's share of the memory budget;
  - a batch runs on one of several lanes (a handle with its own workspace and
    CUDA stream), so frames that arrive while another batch is on the GPU are
    admitted into the next batch on a free lane and overlap on the device;
  - inputs are copied from pinned host memory on the lane's stream, the
    disparity maps are copied back into pinned host buffers, and a completion
    thread resolves each request when its lane's event fires.

Per request the server records arrival and completion times; ``stats()``
gives p50/p99 latency and frames/s.  All matching runs in libdco_stereo.so
(`dco_stereo_match_batch`); this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import threading
import time
from concurrent.futures import Future
from typing import Optional, Sequence

import numpy as np

from .binding import Params, Stereo, Tile


@dataclasses.dataclass
class _Request:
    stream: int
    left: object            # pinned host tensor (H, W, 3) uint8
    right: object
    arrival: float          # time.perf_counter() of the request
    future: Future
    slot: int = -1
    done: float = 0.0
    launch: float = 0.0     # when its batch was enqueued


class _Slot:
    def __init__(self, torch, dev, W, H):
        self.left = torch.empty((H, W, 3), dtype=torch.uint8, device=dev)
        self.right = torch.empty_like(self.left)
        self.out = torch.empty((H, W), dtype=torch.int16, device=dev)
        self.host_out = torch.empty((H, W), dtype=torch.int16).pin_memory()
        self.busy = False


class _Lane:
    def __init__(self, torch, dev, device_index, budget):
        self.stereo = Stereo(device_index, budget)
        self.stream = torch.cuda.Stream(dev)
        self.busy = False


class Server:
    def __init__(self, shapes: Sequence[tuple[int, int, int]], budget_bytes: Optional[int] = None,
                 lanes: int = 2, slots_per_stream: int = 3, max_batch: int = 16,
                 params: Optional[Params] = None, device: int = 0,
                 tiles: Optional[Sequence] = None):
        import torch
        self.torch = torch
        self.dev = torch.device(f"cuda:{device}")
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.params = params
        self.max_batch = max_batch
        # each stream's tiles (e.g. tune.tune_batch); 0 fields = the params' own
        self.tiles = [Tile.of(v) for v in (tiles or [None] * len(self.shapes))]

        def ws_of(s):
            W, H, D = self.shapes[s]
            p = Params.default(**{f: getattr(params, f) for f, _ in Params._fields_}) if params else Params.default()
            return Stereo.workspace_bytes(W, H, D, self.tiles[s].apply(p))
        ws = [ws_of(s) for s in range(len(self.shapes))]
        if budget_bytes is None:
            budget_bytes = lanes * sum(ws)   # every stream can be in every lane's batch
        self.lane_budget = budget_bytes // lanes
        if max(ws) > self.lane_budget:
            raise ValueError("the memory budget cannot hold one frame of the largest stream")
        self.ws = ws
        self.slots = [[_Slot(torch, self.dev, W, H) for _ in range(slots_per_stream)]
                      for (W, H, _) in self.shapes]
        self.lanes = [_Lane(torch, self.dev, device, self.lane_budget) for _ in range(lanes)]
        # warm every lane up with the largest batch admission allows, so its
        # workspace never grows (a synchronising reallocation) while serving
        warm, used = [], 0
        for s, (W, H, D) in enumerate(self.shapes):
            for sl in self.slots[s]:
                if used + ws[s] <= self.lane_budget and len(warm) < max_batch:
                    warm.append((sl.left, sl.right, D, sl.out, self.tiles[s]))
                    used += ws[s]
        for sl_list in self.slots:
            for sl in sl_list:
                sl.left.zero_()
                sl.right.zero_()
        for ln in self.lanes:
            ln.stereo.match_batch(warm, params, stream=torch.cuda.current_stream(self.dev))
        torch.cuda.synchronize(self.dev)
        self.pending = collections.deque()
        self.cv = threading.Condition()
        self.inflight = collections.deque()
        self.done_cv = threading.Condition()
        self.records = []
        self.stop = False
        self.sched = threading.Thread(target=self._schedule, daemon=True)
        self.compl = threading.Thread(target=self._complete, daemon=True)
        self.sched.start()
        self.compl.start()

    # ------------------------------------------------------------ client side
    def submit(self, stream: int, left, right, arrival: Optional[float] = None) -> Future:
        """Queue one frame of `stream` (pinned host uint8 tensors (H, W, 3))."""
        fut = Future()
        req = _Request(stream, left, right, time.perf_counter() if arrival is None else arrival, fut)
        with self.cv:
            self.pending.append(req)
            self.cv.notify_all()
        return fut

    def close(self) -> None:
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self.sched.join()
        with self.done_cv:
            self.done_cv.notify_all()
        self.compl.join()
        self.torch.cuda.synchronize(self.dev)
        for ln in self.lanes:
            ln.stereo.close()

    def stats(self) -> dict:
        lat = np.array([r[3] - r[2] for r in self.records]) * 1e3
        if lat.size == 0:
            return {"frames": 0}
        t0 = min(r[2] for r in self.records)
        t1 = max(r[3] for r in self.records)
        per = {}
        for s in range(len(self.shapes)):
            ls = np.array([r[3] - r[2] for r in self.records if r[0] == s]) * 1e3
            if ls.size:
                per[s] = {"frames": int(ls.size), "p50_ms": float(np.percentile(ls, 50)),
                          "p99_ms": float(np.percentile(ls, 99))}
        # where the latency goes: arrival -> batch enqueued (admission and
        # scheduling), the batch's device time (input copies, match, map
        # copies), and the rest (host launch overhead, completion hand-off)
        queue = np.array([r[4] - r[2] for r in self.records]) * 1e3
        gpu = np.array([r[5] for r in self.records])
        rest = lat - queue - gpu
        parts = {k: {"p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
                 for k, v in (("queue", queue), ("device", gpu), ("host_rest", rest))}
        return {"frames": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "frames_per_s": lat.size / max(t1 - t0, 1e-9),
                "batches": self.n_batches, "mean_batch": self.n_frames_batched / max(self.n_batches, 1),
                "per_stream": per, "latency_parts": parts}

    # ----------------------------------------------------------- scheduling
    n_batches = 0
    n_frames_batched = 0
    max_batch_bytes = 0   # largest workspace a formed batch needed

    def _free_slot(self, stream: int) -> int:
        for i, sl in enumerate(self.slots[stream]):
            if not sl.busy:
                return i
        return -1

    def _form_batch(self):
        """Admit pending requests in arrival order while a slot and memory are free."""
        batch, used, skipped = [], 0, collections.deque()
        while self.pending and len(batch) < self.max_batch:
            req = self.pending.popleft()
            si = self._free_slot(req.stream)
            need = self.ws[req.stream]
            if si < 0 or used + need > self.lane_budget:
                skipped.append(req)
                continue
            req.slot = si
            self.slots[req.stream][si].busy = True
            used += need
            batch.append(req)
        self.max_batch_bytes = max(self.max_batch_bytes, used)
        while skipped:   # keep arrival order for the ones left behind
            self.pending.appendleft(skipped.pop())
        return batch

    def _schedule(self):
        torch = self.torch
        while True:
            with self.cv:
                while not self.stop and not (self.pending and any(not ln.busy for ln in self.lanes)):
                    self.cv.wait(0.05)
                if self.stop and not self.pending:
                    break
                lane = next((ln for ln in self.lanes if not ln.busy), None)
                if lane is None:
                    continue
                batch = self._form_batch()
                if not batch:
                    self.cv.wait(0.001)
                    continue
                lane.busy = True
            try:
                with torch.cuda.stream(lane.stream):
                    pairs = []
                    for r in batch:
                        sl = self.slots[r.stream][r.slot]
                        sl.left.copy_(r.left, non_blocking=True)
                        sl.right.copy_(r.right, non_blocking=True)
                        pairs.append((sl.left, sl.right, self.shapes[r.stream][2], sl.out, self.tiles[r.stream]))
                    t_launch = time.perf_counter()
                    ev0 = torch.cuda.Event(enable_timing=True)
                    ev0.record(lane.stream)
                    lane.stereo.match_batch(pairs, self.params, stream=lane.stream)
                    for r in batch:
                        sl = self.slots[r.stream][r.slot]
                        sl.host_out.copy_(sl.out, non_blocking=True)
                    ev = torch.cuda.Event(enable_timing=True)
                    ev.record(lane.stream)
                    for r in batch:
                        r.launch = t_launch
            except Exception as exc:   # fail this batch's requests, keep serving
                lane.stream.synchronize()
                with self.cv:
                    for r in batch:
                        self.slots[r.stream][r.slot].busy = False
                        r.future.set_exception(exc)
                    lane.busy = False
                    self.cv.notify_all()
                continue
            self.n_batches += 1
            self.n_frames_batched += len(batch)
            with self.done_cv:
                self.inflight.append((lane, ev0, ev, batch))
                self.done_cv.notify_all()

    def _complete(self):
        while True:
            with self.done_cv:
                while not self.inflight and not (self.stop and not self.sched.is_alive()):
                    self.done_cv.wait(0.05)
                if not self.inflight:
                    if self.stop and not self.sched.is_alive():
                        break
                    continue
                lane, ev0, ev, batch = self.inflight.popleft()
            ev.synchronize()
            t = time.perf_counter()
            gpu_ms = ev0.elapsed_time(ev)   # copies in, match, copies out on the lane's stream
            for r in batch:
                sl = self.slots[r.stream][r.slot]
                r.done = t
                r.future.set_result(sl.host_out.numpy().copy())
                self.records.append((r.stream, r.slot, r.arrival, t, r.launch, gpu_ms))
            with self.cv:
                for r in batch:
                    self.slots[r.stream][r.slot].busy = False
                lane.busy = False
                self.cv.notify_all()


def _stream_frames(i: int, W: int, H: int, D: int, n: int):
    from . import scenes
    st = scenes.StreamScene(i, W, H, D)
    return [(s.left, s.right) for s in (st.frame(t) for t in range(n))]


def render_frames(shapes, n: int, processes: int = 0):
    """`n` consecutive frames of every stream (planes moving 0-3 px per frame),
    as pinned host tensors: frames[stream][t] = (left, right).  processes > 0
    renders the streams in a spawned process pool (safe after CUDA set-up)."""
    import torch
    jobs = [(i, W, H, D, n) for i, (W, H, D) in enumerate(shapes)]
    if processes > 0:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(min(processes, len(jobs)), mp_context=mp.get_context("spawn")) as ex:
            raw = list(ex.map(_stream_frames, *zip(*jobs)))
    else:
        raw = [_stream_frames(*j) for j in jobs]
    return [[(torch.from_numpy(l).pin_memory(), torch.from_numpy(r).pin_memory()) for l, r in fr] for fr in raw]


def run_saturation(duration_s: float = 3.0, shapes=None, unique_frames: int = 4, device: int = 0, server_kw=None,
                   frames=None):
    """Closed loop: every stream keeps `slots_per_stream` frames in flight
    (a new frame is submitted as soon as one of its stream completes), for
    `duration_s` seconds: the server's throughput ceiling, with the latency
    at that load.  Returns the server stats."""
    from . import scenes
    shapes = shapes or scenes.STREAMS_CONFIG4
    frames = frames or render_frames(shapes, unique_frames)
    unique_frames = len(frames[0])
    kw = dict(server_kw or {})
    depth = kw.get("slots_per_stream", 3)
    srv = Server(shapes, device=device, **kw)
    gc.collect()
    gc.disable()
    try:
        t_end = time.perf_counter() + duration_s
        k = [0] * len(shapes)
        live = collections.deque()
        for i in range(len(shapes)):
            for _ in range(depth):
                l, r = frames[i][k[i] % unique_frames]
                live.append((i, srv.submit(i, l, r)))
                k[i] += 1
        while live:
            i, f = live.popleft()
            f.result(timeout=120)
            if time.perf_counter() < t_end:
                l, r = frames[i][k[i] % unique_frames]
                live.append((i, srv.submit(i, l, r)))
                k[i] += 1
    finally:
        gc.enable()
    srv.close()
    return srv.stats()


def run_config4(frames_per_stream: int = 300, rate_hz: float = 30.0, time_scale: float = 1.0,
                unique_frames: int = 6, shapes=None, device: int = 0, server_kw=None, frames=None):
    """Replay config 4: Poisson arrivals per stream, frames cycled from a few
    rendered ones (planes translating 0-3 px/frame).  time_scale > 1 replays
    faster than real time.  Returns (server stats, outputs by (stream, frame))."""
    import torch
    from . import scenes
    shapes = shapes or scenes.STREAMS_CONFIG4
    frames = frames or render_frames(shapes, unique_frames)
    unique_frames = len(frames[0])
    events = []
    for i in range(len(shapes)):
        arr = scenes.poisson_arrivals(frames_per_stream, rate_hz, scenes.seed_for(4, 100 + i))
        events += [(t / time_scale, i, k) for k, t in enumerate(arr)]
    events.sort()
    srv = Server(shapes, device=device, **(server_kw or {}))
    futs = {}
    # a full collection of the Python heap mid-replay pauses every thread of
    # the serving loop at once: collect before the replay, not during it
    gc.collect()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for t, i, k in events:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            l, r = frames[i][k % unique_frames]
            futs[(i, k)] = srv.submit(i, l, r, arrival=t0 + t)
        outs = {key: f.result(timeout=120) for key, f in futs.items()}
    finally:
        gc.enable()
    srv.close()
    return srv.stats(), outs, frames


# ------------------------------------------------------------ native runtime
def _native_stats(records, nstreams: int, counters: dict) -> dict:
    """records: (stream, arrival_s, launch_s, done_s, device_ms) per frame."""
    lat = np.array([r[3] - r[1] for r in records]) * 1e3
    if lat.size == 0:
        return {"frames": 0}
    queue = np.array([r[2] - r[1] for r in records]) * 1e3
    dev = np.array([r[4] for r in records])
    rest = lat - queue - dev
    t0 = min(r[1] for r in records)
    t1 = max(r[3] for r in records)
    per = {}
    for s in range(nstreams):
        ls = np.array([r[3] - r[1] for r in records if r[0] == s]) * 1e3
        if ls.size:
            per[s] = {"frames": int(ls.size), "p50_ms": float(np.percentile(ls, 50)),
                      "p99_ms": float(np.percentile(ls, 99))}
    parts = {k: {"p50_ms": float(np.percentile(v, 50)), "p99_ms": float(np.percentile(v, 99))}
             for k, v in (("queue", queue), ("device", dev), ("host_rest", rest))}
    return {"frames": int(lat.size), "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "frames_per_s": lat.size / max(t1 - t0, 1e-9), "batches": counters["batches"],
            "mean_batch": counters["frames"] / max(counters["batches"], 1), "per_stream": per,
            "latency_parts": parts, "runtime": "native"}


def run_config4_native(frames_per_stream: int = 300, rate_hz: float = 30.0, time_scale: float = 1.0,
                       unique_frames: int = 6, shapes=None, device: int = 0, frames=None, tiles=None,
                       keep_outputs: bool = False, server_kw=None):
    """Config 4 replayed through the library's native serving runtime
    (dco_server_*): Poisson arrivals per stream, each frame's map copied by
    the server straight into a pinned output buffer.  Returns (stats,
    outputs by (stream, frame) if keep_outputs, frames)."""
    import torch
    from . import scenes
    from .binding import NativeServer
    shapes = shapes or scenes.STREAMS_CONFIG4
    frames = frames or render_frames(shapes, unique_frames)
    unique_frames = len(frames[0])
    events = []
    for i in range(len(shapes)):
        arr = scenes.poisson_arrivals(frames_per_stream, rate_hz, scenes.seed_for(4, 100 + i))
        events += [(t / time_scale, i, k) for k, t in enumerate(arr)]
    events.sort()
    kw = dict(server_kw or {})
    slots = kw.get("slots_per_stream", 3)
    # output buffers: every frame its own when kept, else a ring per stream
    # deeper than the frames a stream can have in flight
    ring = 4 * slots

    def out_buf(i, k):
        W, H, _ = shapes[i]
        return torch.empty((H, W), dtype=torch.int16).pin_memory().numpy()
    outs = {} if keep_outputs else {(i, j): out_buf(i, j) for i in range(len(shapes)) for j in range(ring)}
    srv = NativeServer(shapes, device=device, tiles=tiles, **kw)
    tickets = [collections.deque() for _ in shapes]   # per stream, oldest first
    records = []

    def retire(i):
        tm = srv.wait(tickets[i].popleft())
        records.append((i, tm.arrival_s, tm.launch_s, tm.done_s, tm.device_ms))
    gc.collect()
    gc.disable()
    try:
        t0 = time.perf_counter()
        for t, i, k in events:
            now = time.perf_counter() - t0
            if t > now:
                time.sleep(t - now)
            while len(tickets[i]) >= ring:   # the ring buffer about to be reused is free
                retire(i)
            l, r = frames[i][k % unique_frames]
            if keep_outputs:
                outs[(i, k)] = out_buf(i, k)
                o = outs[(i, k)]
            else:
                o = outs[(i, k % ring)]
            tickets[i].append(srv.submit(i, l.numpy(), r.numpy(), o))
        for i in range(len(shapes)):
            while tickets[i]:
                retire(i)
    finally:
        gc.enable()
    cnt = srv.counters()
    srv.close()
    return _native_stats(records, len(shapes), cnt), (outs if keep_outputs else None), frames


def run_saturation_native(duration_s: float = 3.0, shapes=None, unique_frames: int = 4, device: int = 0,
                          frames=None, tiles=None, server_kw=None):
    """Closed loop through the native runtime: every stream keeps its slots
    busy (a new frame as soon as one of the stream completes) for
    `duration_s` seconds."""
    import torch
    from . import scenes
    from .binding import NativeServer
    shapes = shapes or scenes.STREAMS_CONFIG4
    frames = frames or render_frames(shapes, unique_frames)
    unique_frames = len(frames[0])
    kw = dict(server_kw or {})
    depth = kw.get("slots_per_stream", 3)
    srv = NativeServer(shapes, device=device, tiles=tiles, **kw)
    bufs = {(i, j): torch.empty((shapes[i][1], shapes[i][0]), dtype=torch.int16).pin_memory().numpy()
            for i in range(len(shapes)) for j in range(depth)}
    records = []
    gc.collect()
    gc.disable()
    try:
        t_end = time.perf_counter() + duration_s
        k = [0] * len(shapes)
        live = collections.deque()
        for i in range(len(shapes)):
            for j in range(depth):
                l, r = frames[i][k[i] % unique_frames]
                live.append((i, j, srv.submit(i, l.numpy(), r.numpy(), bufs[(i, j)])))
                k[i] += 1
        while live:
            i, j, tk = live.popleft()
            tm = srv.wait(tk)
            records.append((i, tm.arrival_s, tm.launch_s, tm.done_s, tm.device_ms))
            if time.perf_counter() < t_end:
                l, r = frames[i][k[i] % unique_frames]
                live.append((i, j, srv.submit(i, l.numpy(), r.numpy(), bufs[(i, j)])))
                k[i] += 1
    finally:
        gc.enable()
    cnt = srv.counters()
    srv.close()
    return _native_stats(records, len(shapes), cnt)
