#!/usr/bin/env python
"""Benchmark of the AD-census matcher (arXiv 2203.02300, Sect. 4) on GB300.

Workload: one rectified RGB pair, 640x480, D = 64 (seeded synthetic scene of
12 slanted planes, Gaussian noise sigma 2, right view gain 1.03 offset +5).
A step is one pass of the whole path on that pair: grey/census/arms for both
views, Eq. 1 costs, Eq. 2 aggregation, Eq. 3 WTA for both reference views,
left-right check.  Metric: disparity evaluations per second, W*H*D per pair.

Own arm (default): inputs resident in HBM; the L2 (129 MB) is flushed by a
256 MiB write between timed steps (outside the step's CUDA events); steps are
timed with CUDA events on the launching stream.  Under torchrun each rank
runs an independent replica on its own GPU (no collective on the data path);
the total is divided by the slowest rank's time.

--impl reference: the FP64 CPU oracle, on the host cores, on bounded row
samples of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

W, H, D = 640, 480, 64
CONFIG = {"workload": "single rectified RGB pair 640x480 D=64, 12 slanted planes, noise sigma 2, "
                      "right gain 1.03 offset +5 (seeded synthetic)",
          "W": W, "H": H, "D": D, "views": 2, "lr_check": True,
          "l2": "flushed between timed steps (device and end-to-end) by a 256 MiB write outside the timed calls"}
METRIC = "disparity evals/sec (W*H*D per pair per second) at 640x480 D=64"
UNIT = "evals/s"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--d-chunk", type=int, default=0, help="fixed pass width instead of the autotuner's")
    ap.add_argument("--tile", default="", help="fixed tile d_chunk,h_chunk,v_chunk instead of the autotuner's")
    ap.add_argument("--no-extras", action="store_true", help="skip the config 3 batch and config 4 serving runs")
    ap.add_argument("--extras", default="all",
                    help="comma list of the extra measurements to run (vote_config2, depth_1280x720, "
                         "smooth_config2, vh_order_config2, densify_1280x720, batch_config3, batch_config5, "
                         "serve_config4), or all")
    return ap.parse_args()


def dist_env():
    from paper_2203_02300_gb300 import replicas
    return replicas.rank_env()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return PEAKS_FALLBACK, "fallback"


MATCHER_SOURCES = ("dco_stereo.cu", "kernels.cuh")   # the files that define the matcher's kernels


def source_digest() -> str:
    """Digest of the matcher's device code and launch geometry without
    comments, stamped into the ncu summaries under profiles/ (a summary of
    other code is not used).  It covers kernels.cuh, the device part of
    dco_stereo.cu (everything before its host section) and the geometry
    functions that size the launches; changes of comments, includes or other
    host code keep it."""
    def strip(code: str) -> str:
        code = re.sub(r"/\*.*?\*/", "", code, flags=re.S)
        code = re.sub(r"//[^\n]*", "", code)
        return "\n".join(l.rstrip() for l in code.splitlines() if l.strip() and not l.startswith("#include"))
    csrc = os.path.join(ROOT, "paper_2203_02300_gb300", "csrc")
    with open(os.path.join(csrc, "kernels.cuh")) as fh:
        parts = [fh.read()]
    with open(os.path.join(csrc, "dco_stereo.cu")) as fh:
        cu = fh.read()
    host = cu.index("// ====================================================================== host")
    parts.append(cu[:host])
    parts.append(cu[cu.index("struct HGeom {"):cu.index("// ---- TMA tile maps")])
    h = hashlib.sha256()
    for part in parts:
        h.update(strip(part).encode())
    return h.hexdigest()[:16]


def ncu_figure(kernel: str, key: str):
    """A per-launch figure (`key: value` line) of `kernel` from the committed
    ncu summary, if that summary was taken on the current kernel source
    (else None)."""
    dig = source_digest()
    for path in glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_*.md")):
        text = open(path).read()
        m = re.search(r"source_digest:\s*(\w+)", text)
        t = re.search(key + r":\s*([0-9.eE+]+)", text)
        if m and t and m.group(1) == dig:
            return float(t.group(1))
    return None


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` (dram__bytes_read.sum + write.sum)."""
    return ncu_figure(kernel, "traffic_bytes_per_launch")


# ------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi samples during the timed region (every 200 ms)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.idx), "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except OSError:
            rows = []
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [c.strip() for c in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if sm:
            res = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return res


# --------------------------------------------------------------- own arm
# Algorithmic HBM bytes of each kernel per launch (what the method must move:
# inputs read once, outputs written once).  npx = W*H, ev = view-evaluations
# of the pass (2 views * npx * disparities of the pass).
def algorithmic_bytes(kernel: str, npx: int, ev_pass: int, npass: int) -> float:
    if kernel == "k_pack":
        return 2 * npx * (3 + 4 + 1)                       # rgb in, rgbx + grey out
    if kernel == "k_prep":
        return 2 * npx * (4 + 1 + 16 + 4)                  # rgbx + grey in, record + arms out
    if kernel == "k_hagg":
        return 4 * ev_pass + 2 * npx * (16 + 16 + 4)       # slice out; records + arms in
    if kernel == "k_vagg":
        return 4 * ev_pass + 2 * npx * (4 + 2 + (16 if npass > 1 else 0))   # slice in; arms in, disparity/state out
    if kernel == "k_lr":
        return npx * (2 + 2 + 2)
    return 0.0


def own_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import __graft_entry__
    from paper_2203_02300_gb300 import binding, replicas, scenes, tune

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    dev = torch.device(f"cuda:{local_rank}")
    s = scenes.config_scene(2)
    Lh = torch.from_numpy(s.left).pin_memory()
    Rh = torch.from_numpy(s.right).pin_memory()
    L = Lh.to(dev)
    R = Rh.to(dev)
    out = torch.empty((H, W), dtype=torch.int16, device=dev)
    st = binding.Stereo(local_rank)
    if args.tile:
        tile = binding.Tile.of([int(v) for v in args.tile.split(",")])
    elif args.d_chunk > 0 or args.no_tune:
        tile = binding.Tile(args.d_chunk)
    else:
        tile = tune.tune_tiles(st, L, R, D)
    dchunk = tile.d_chunk
    p = tile.apply(binding.Params.default())
    npass = -(-D // (dchunk or D))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(max(args.warmup, 3)):
        st.match(L, R, D, p, out)
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps, L2 flushed between steps
    clocks = Clocks(local_rank if torch.cuda.device_count() > 1 else 0)
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    launches0 = st.launch_count()
    t_wall0 = time.perf_counter()
    for a, b in evs:
        flush.zero_()
        a.record(stream)
        st.match(L, R, D, p, out)
        b.record(stream)
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    launches = st.launch_count() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    units, total_s, value = replicas.job_rate(W * H * D * args.steps, total_ms * 1e-3, dist, dev)
    total_ms = total_s * 1e3

    # ---- end to end: host buffers through the C ABI (copies inside)
    Ln, Rn = Lh.numpy(), Rh.numpy()
    outh = torch.empty((H, W), dtype=torch.int16).pin_memory().numpy()
    for _ in range(3):
        st.match_host(Ln, Rn, D, p, out=outh)
    e2e_ms = []
    for _ in range(args.steps):
        flush.zero_()   # L2 flushed between steps here too, outside the timed call
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st.match_host(Ln, Rn, D, p, out=outh)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    _, _, e2e_value = replicas.job_rate(W * H * D * args.steps, sum(e2e_ms) * 1e-3, dist, dev)
    check = st.match(L, R, D, p, out)
    torch.cuda.synchronize(dev)
    assert np.array_equal(outh, check.cpu().numpy()), "host path differs from device path"

    # ---- per-kernel durations (library CUDA events on the same stream)
    st.set_profiling(True)
    st.profile_reset()
    for _ in range(args.steps):
        flush.zero_()
        st.match(L, R, D, p, out)
    torch.cuda.synchronize(dev)
    prof = st.profile()
    st.set_profiling(False)
    npx = W * H
    dc = dchunk or D
    kernels = {}
    for k, (n, ms) in prof.items():
        avg = ms / n
        ev_pass = 2 * npx * dc
        kernels[k] = {"launches": n, "avg_us": round(avg * 1e3, 3),
                      "share": None, "alg_bytes": algorithmic_bytes(k, npx, ev_pass, npass)}
    ktot = sum(v["avg_us"] * v["launches"] for v in kernels.values())
    for v in kernels.values():
        v["share"] = round(v["avg_us"] * v["launches"] / ktot, 4)
    dom = max(kernels, key=lambda k: kernels[k]["avg_us"] * kernels[k]["launches"])
    pk, src = peaks()
    achieved = kernels[dom]["alg_bytes"] / (kernels[dom]["avg_us"] * 1e-6) / 1e9
    roof = {"kernel": dom, "bound": "hbm", "achieved": round(achieved, 1), "peak": pk["hbm_gbs"],
            "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 4),
            "traffic": ncu_traffic(dom), "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"
            if src == "measured" else "fallback 6.8 TB/s"}
    # the on-chip pipe that binds the dominant kernel: shared-memory data
    # wavefronts (one 128-byte wavefront per SM per cycle) from the committed
    # ncu summary, over the live duration, against SMs x the sampled SM clock
    wf = ncu_figure(dom, "shared_wavefronts_per_launch")
    if wf and clk.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        ach = wf / (kernels[dom]["avg_us"] * 1e-6) / 1e9
        pk_wf = sms * clk["sm_mhz"] * 1e-3
        roof["on_chip"] = {"pipe": "L1 shared-memory data path", "achieved": round(ach, 1), "peak": round(pk_wf, 1),
                           "unit": "G wavefronts/s", "frac": round(ach / pk_wf, 4),
                           "wavefronts_per_launch": int(wf), "peak_source": f"{sms} SMs x {clk['sm_mhz']} MHz"}

    # ---- the cost + aggregation kernels together (Eq. 1-3: k_hagg, k_vagg):
    # their algorithmic bytes over their summed time, against the same peak
    hv = [k for k in ("k_hagg", "k_vagg") if k in kernels]
    hv_us = sum(kernels[k]["avg_us"] * kernels[k]["launches"] for k in hv) / args.steps
    hv_bytes = sum(kernels[k]["alg_bytes"] * kernels[k]["launches"] for k in hv) / args.steps
    costagg = {"kernels": hv, "us_per_frame": round(hv_us, 2), "alg_bytes_per_frame": hv_bytes,
               "achieved_gbs": round(hv_bytes / (hv_us * 1e-6) / 1e9, 1) if hv_us > 0 else None,
               "frac_hbm": round(hv_bytes / (hv_us * 1e-6) / 1e9 / pk["hbm_gbs"], 4) if hv_us > 0 else None}

    # ---- config 3 (batched) and config 4 (serving), rank 0 only
    extras = {}
    want = set() if args.no_extras else {e.strip() for e in args.extras.split(",") if e.strip()}
    on = (lambda name: "all" in want or name in want)
    if rank == 0:
        if on("vote_config2"):
            extras["vote_config2"] = vote_config2(torch, binding, st, L, R, D, dchunk, flush, dev)
        if on("depth_1280x720"):
            extras["depth_1280x720"] = depth_full_size(torch, binding, st, flush, dev)
        if on("smooth_config2"):
            extras["smooth_config2"] = smooth_config2(torch, binding, st, L, R, D, dchunk, flush, dev)
        if on("vh_order_config2"):
            extras["vh_order_config2"] = vh_order_config2(torch, binding, st, L, R, D, dchunk, flush, dev)
        if on("densify_1280x720"):
            extras["densify_1280x720"] = densify_full_size(torch, binding, st, flush, dev)
        if on("batch_config3"):
            extras["batch_config3"] = batch_config3(torch, binding, st, flush, dev)
        if on("batch_config5"):
            extras["batch_config5"] = batch_config5(torch, binding, flush, dev)
        if on("serve_config4"):
            from paper_2203_02300_gb300.serve import render_frames
            frames4 = render_frames(scenes.STREAMS_CONFIG4, 16, processes=4)
            d4 = tune.tune_batch(st, scenes.STREAMS_CONFIG4, device=local_rank)
            # the smaller streams latency-critical (shortest job first), and
            # the same replay with every stream in plain arrival order
            extras["serve_config4"] = serve_config4_native(torch, binding, st, local_rank, frames=frames4,
                                                           tiles=d4, priorities="smaller")
            extras["serve_config4_fifo"] = serve_config4_native(torch, binding, st, local_rank, frames=frames4,
                                                                tiles=d4)
            extras["serve_config4_5x_rate"] = serve_config4_native(torch, binding, st, local_rank, time_scale=5.0,
                                                                   frames=frames4, tiles=d4, priorities="smaller")
            extras["serve_config4_saturation"] = serve_saturation(torch, local_rank, frames4, d4)
            # the same replay through the Python serving loop, with the plain
            # single calls of each size and the served == alone check
            extras["serve_config4_python_loop"] = serve_config4(torch, binding, st, local_rank, frames=frames4,
                                                                tiles=d4)

    # ---- CPU baseline: the oracle on the host cores (rank 0, N = 1)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = oracle_rate(s, budget_s=12.0)

    if rank == 0:
        lat = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 cost, u32 fixed-point aggregation",
            "data": "synthetic (seeded plane scene; the paper's INDEMIND / Middlebury data are not available)",
            "config": dict(CONFIG, d_chunk=dc, h_chunk=tile.h_chunk, v_chunk=tile.v_chunk, passes=npass,
                           parallelism=f"replicas x{world}"),
            "frames_per_s": 1e3 * args.steps * world / total_ms,
            "latency_ms": {"p50": statistics.median(lat), "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * W * H * 3,
                    "d2h_bytes_per_step": W * H * 2,
                    "latency_ms": {"p50": statistics.median(e2e_ms),
                                   "p99": sorted(e2e_ms)[min(len(e2e_ms) - 1, int(0.99 * len(e2e_ms)))]}},
            "roofline": roof,
            "cost_aggregation": costagg,
            "kernels": kernels,
            "gpu_launches": launches,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                       "samples": clk["samples"]},
            "wall_s_timed_region": t_wall,
            "cpu_baseline": cpu,
        }
        line.update(extras)
        print(json.dumps(line))
    st.close()
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------- Eq. 4 rounds (config 2)
def vote_config2(torch, binding, st, L, R, D, dchunk, flush, dev, reps: int = 20, rounds: int = 2):
    """The config 2 path with `rounds` Eq. 4 rounds against the path without,
    and the vote kernels' own durations (library CUDA events, L2 flushed
    before every call) against their algorithmic bytes."""
    W, H = L.shape[1], L.shape[0]
    npx = W * H
    out = torch.empty((H, W), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)

    def med_ms(p):
        for _ in range(3):
            st.match(L, R, D, p, out)
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st.match(L, R, D, p, out)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    p0 = binding.Params.default(d_chunk=dchunk)
    pv = binding.Params.default(d_chunk=dchunk, vote_iters=rounds)
    t0, tv = med_ms(p0), med_ms(pv)
    st.set_profiling(True)
    st.profile_reset()
    for _ in range(reps):
        flush.zero_()
        st.match(L, R, D, pv, out)
    torch.cuda.synchronize(dev)
    prof = st.profile()
    st.set_profiling(False)
    pk, _ = peaks()
    dc = dchunk or D
    alg = {"k_hvote": lambda: npx * (2 + 4) + 4 * npx * dc,        # map + arms in, count slice out
           "k_vvote": lambda: 4 * npx * dc + npx * (4 + 2 + 2)}   # slice + arms + mask in, map out
    kern = {}
    round_us = 0.0
    for k in ("k_hvote", "k_vvote"):
        if k not in prof:
            continue
        n, ms = prof[k]
        avg_us = ms / n * 1e3
        round_us += avg_us * n / (reps * rounds)
        gbs = alg[k]() / (avg_us * 1e-6) / 1e9
        kern[k] = {"launches_per_round": n / (reps * rounds), "avg_us": round(avg_us, 3),
                   "achieved_gbs": round(gbs, 1), "frac_hbm": round(gbs / pk["hbm_gbs"], 4)}
    return {"rounds": rounds, "ms_path": round(t0, 4), "ms_path_with_rounds": round(tv, 4),
            "us_per_round": round(round_us, 2),
            "votes_per_s": npx * D / (round_us * 1e-6) if round_us else None,
            "kernels": kern}


# ------------------------------------ arm smoothing, Sect. 4.1 (config 2)
def smooth_config2(torch, binding, st, L, R, D, dchunk, flush, dev, reps: int = 20):
    """The config 2 path with the smoothed cross-support window against the
    path without; the smoothing kernel's duration against its bytes."""
    W, H = L.shape[1], L.shape[0]
    out = torch.empty((H, W), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)

    def med_ms(p):
        for _ in range(3):
            st.match(L, R, D, p, out)
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st.match(L, R, D, p, out)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    p1 = binding.Params.default(d_chunk=dchunk, smooth_arms=1)
    t0, t1 = med_ms(binding.Params.default(d_chunk=dchunk)), med_ms(p1)
    st.set_profiling(True)
    st.profile_reset()
    for _ in range(reps):
        flush.zero_()
        st.match(L, R, D, p1, out)
    torch.cuda.synchronize(dev)
    n, ms = st.profile().get("k_smooth", (0, 0.0))
    st.set_profiling(False)
    pk, _ = peaks()
    avg = ms / n * 1e3 if n else None
    alg = 2 * W * H * (4 + 4) + W * H * 8   # per pass: arms in/out (both images); records touched once
    return {"ms_path": round(t0, 4), "ms_path_smoothed": round(t1, 4),
            "k_smooth": {"launches_per_frame": n / reps, "avg_us": round(avg, 3) if avg else None,
                         "frac_hbm": round(alg / (avg * 1e-6) / 1e9 / pk["hbm_gbs"], 4) if avg else None}}


# ----------------- the other aggregation order, Sect. 4.2.2 (config 2)
def vh_order_config2(torch, binding, st, L, R, D, dchunk, flush, dev, reps: int = 20):
    """The config 2 path with vertical sums first (k_vcost, then the row scan
    k_hwta) against the default order; per-kernel CUDA-event averages."""
    W, H = L.shape[1], L.shape[0]
    out = torch.empty((H, W), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, order in (("hv", 0), ("vh", 1)):
        p = binding.Params.default(d_chunk=dchunk, agg_order=order)
        for _ in range(3):
            st.match(L, R, D, p, out)
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st.match(L, R, D, p, out)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        st.set_profiling(True)
        st.profile_reset()
        for _ in range(reps):
            flush.zero_()
            st.match(L, R, D, p, out)
        torch.cuda.synchronize(dev)
        prof = st.profile()
        st.set_profiling(False)
        res[f"ms_path_{name}"] = round(statistics.median(ts), 4)
        for k in (("k_hagg", "k_vagg") if order == 0 else ("k_vcost", "k_hwta")):
            n, ms = prof.get(k, (0, 0.0))
            res[f"{k}_us"] = round(ms / n * 1e3, 3) if n else None
    return res


# --------------------------------------------- densification (Sect. 6)
def densify_full_size(torch, binding, st, flush, dev, W: int = 1280, H: int = 720, reps: int = 5):
    """Eq. 20 on a 1280x720 frame: the sparse depth of the quarter-size path,
    a depth contour where the ground truth jumps, texture weights from the
    image gradient (M_fuse = 1).  Median time per solve and iterations with
    the one-launch solve (solver 0) and with two launches per iteration
    (solver 1, whose two streaming kernels are set against their algorithmic
    bytes)."""
    import numpy as np
    from paper_2203_02300_gb300 import scenes
    s = scenes.plane_scene(W, H, 128, 12, seed=scenes.seed_for(2, 950), drange=(4, 120), slanted=True,
                           noise_sigma=2.0)
    L = torch.from_numpy(s.left).to(dev)
    R = torch.from_numpy(s.right).to(dev)
    z = st.depth(L, R, 64, 700.0, 0.12)
    g = s.disp
    B = ((np.abs(np.diff(g, axis=1, append=g[:, -1:])) > 1) | (np.abs(np.diff(g, axis=0, append=g[-1:])) > 1))
    Y = s.left.astype(np.float32).mean(axis=2)
    gm = np.hypot(*np.gradient(Y))
    Bd = torch.from_numpy(B.astype(np.uint8)).to(dev)
    mi = torch.from_numpy((gm / gm.max()).astype(np.float32)).to(dev)
    mf = torch.ones_like(mi)
    out = torch.empty_like(z)
    stream = torch.cuda.current_stream(dev)
    pk, _ = peaks()
    n = W * H
    alg = {"k_dn_ap": 4 * n * 7, "k_dn_upd": 4 * n * 8}   # ap: z, p, wr, wd, diag in; p, Ap out. upd: x, p, r, Ap, diag in; x, r, z out
    res = {"size": f"{W}x{H}", "sparse_fraction": float((z > 0).float().mean().item())}
    for solver in (0, 1):
        p = binding.DenseParams.default(solver=solver)
        st.densify(z, Bd, mf, mi, None, p, out=out)
        ts = []
        for _ in range(reps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            st.densify(z, Bd, mf, mi, None, p, out=out)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        iters, rel = st.densify_stats()
        st.set_profiling(True)
        st.profile_reset()
        st.densify(z, Bd, mf, mi, None, p, out=out)
        torch.cuda.synchronize(dev)
        prof = st.profile()
        st.set_profiling(False)
        kern = {}
        for k, (cnt, ms) in prof.items():
            avg = ms / cnt * 1e3
            e = {"launches": cnt, "avg_us": round(avg, 3)}
            if k in alg:
                gbs = alg[k] / (avg * 1e-6) / 1e9
                e.update(achieved_gbs=round(gbs, 1), frac_hbm=round(gbs / pk["hbm_gbs"], 4))
            kern[k] = e
        med = statistics.median(ts)
        r = {"iterations": iters, "rel_residual": rel, "tol": float(p.tol), "ms_per_solve": round(med, 3),
             "us_per_iteration": round(1e3 * med / max(iters, 1), 2), "kernels": kern}
        if solver == 0:
            res.update(r)
        else:
            res["per_iteration_launches"] = r
    return res


# ------------------------------------------- quarter size + depth (Sect. 4.4)
def depth_full_size(torch, binding, st, flush, dev, W: int = 1280, H: int = 720, D: int = 64, reps: int = 20):
    """A 1280x720 pair (the sensor size the paper reduces by a quarter):
    downscale to 640x360, match over D = 64 half-size disparities, depth on
    the full grid.  Median CUDA-event time per frame (L2 flushed before each)
    and the two new kernels against their algorithmic bytes."""
    from paper_2203_02300_gb300 import scenes
    s = scenes.plane_scene(W, H, 2 * D, 12, seed=scenes.seed_for(2, 900), drange=(4, 2 * D - 8),
                           slanted=True, slope=0.2, noise_sigma=2.0)
    L = torch.from_numpy(s.left).to(dev)
    R = torch.from_numpy(s.right).to(dev)
    out = torch.empty((H, W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(3):
        st.depth(L, R, D, 700.0, 0.12, out=out)
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.depth(L, R, D, 700.0, 0.12, out=out)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    st.set_profiling(True)
    st.profile_reset()
    for _ in range(reps):
        flush.zero_()
        st.depth(L, R, D, 700.0, 0.12, out=out)
    torch.cuda.synchronize(dev)
    prof = st.profile()
    st.set_profiling(False)
    pk, _ = peaks()
    npx, nh = W * H, (W // 2) * (H // 2)
    alg = {"k_down": 2 * (3 * npx + 3 * nh), "k_depth": 2 * nh + 4 * npx}
    kern = {}
    for k, (n, ms) in prof.items():
        avg = ms / n * 1e3
        e = {"avg_us": round(avg, 3)}
        if k in alg:
            gbs = alg[k] / (avg * 1e-6) / 1e9
            e.update(achieved_gbs=round(gbs, 1), frac_hbm=round(gbs / pk["hbm_gbs"], 4))
        kern[k] = e
    med = statistics.median(ts)
    return {"input": f"{W}x{H}", "matched_at": f"{W // 2}x{H // 2} D={D}", "ms_per_frame": round(med, 4),
            "frames_per_s": 1e3 / med, "evals_per_s": nh * D / (med * 1e-3),
            "valid_fraction": float((out > 0).float().mean().item()), "kernels": kern}


# ------------------------------------------------- config 3 and config 4
def _timed(torch, dev, flush, fn, reps):
    stream = torch.cuda.current_stream(dev)
    ms = []
    for _ in range(reps + 2):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(b))
    return statistics.median(ms[2:])


def batch_config3(torch, binding, st, flush, dev, reps: int = 10):
    """32 pairs of uneven size: one batched pass (CUDA-graph replay) against
    the same pairs matched one call at a time, both with the library's
    automatic tiles and with each shape's tile (pass width, blocks of the two
    1-D passes) from the autotuner;
    L2 flushed before each."""
    from paper_2203_02300_gb300 import scenes, tune
    from paper_2203_02300_gb300.batch import BatchGraph
    sc = scenes.batch_config3(32)
    shapes = [(s.W, s.H, s.D) for s in sc]
    L = [torch.from_numpy(s.left).to(dev) for s in sc]
    R = [torch.from_numpy(s.right).to(dev) for s in sc]
    outs = [torch.empty((s.H, s.W), dtype=torch.int16, device=dev) for s in sc]
    units = sum(s.W * s.H * s.D for s in sc)
    tuned = tune.tune_batch(st, shapes, device=dev.index or 0)
    g = BatchGraph(binding.Stereo(dev.index or 0), shapes, device=dev.index or 0)
    gt = BatchGraph(binding.Stereo(dev.index or 0), shapes, device=dev.index or 0, tiles=tuned)
    g.load(L, R)
    gt.load(L, R)
    pt = [t.apply(binding.Params.default()) for t in tuned]

    def sequential():
        for l, r, s, o in zip(L, R, sc, outs):
            st.match(l, r, s.D, None, o)

    def sequential_tuned():
        for l, r, s, o, p in zip(L, R, sc, outs, pt):
            st.match(l, r, s.D, p, o)

    t_seq = _timed(torch, dev, flush, sequential, reps)
    t_bat = _timed(torch, dev, flush, g.replay, reps)
    t_seq_t = _timed(torch, dev, flush, sequential_tuned, reps)
    t_bat_t = _timed(torch, dev, flush, gt.replay, reps)
    same = all(torch.equal(a, b) and torch.equal(a, c) for a, b, c in zip(outs, g.out, gt.out))
    sizes = sorted(set(shapes))
    tiles = {f"{w}x{h} D={d}": list(tuned[shapes.index((w, h, d))]) for w, h, d in sizes}
    return {"pairs": len(sc), "sizes": [f"{w}x{h} D={d}" for w, h, d in sizes], "evals": units,
            "batched_graph_ms": t_bat, "batched_evals_per_s": units / (t_bat * 1e-3),
            "sequential_ms": t_seq, "sequential_evals_per_s": units / (t_seq * 1e-3),
            "speedup": t_seq / t_bat,
            "tuned_tiles_d_h_v": tiles,
            "tuned_batched_graph_ms": t_bat_t, "tuned_batched_evals_per_s": units / (t_bat_t * 1e-3),
            "tuned_sequential_ms": t_seq_t, "tuned_sequential_evals_per_s": units / (t_seq_t * 1e-3),
            "tuned_batch_over_default_sequential": t_seq / t_bat_t,
            "identical_to_sequential": bool(same)}


def batch_config5(torch, binding, flush, dev, reps: int = 3, budget: int = 1_500_000_000):
    """8 pairs of 1920x1080, D = 256 in one batched call on a handle whose
    workspace budget is below one 2.12 GB FP32 volume: the library admits the
    pairs in groups that fit (passes of 32 disparities), the allocation
    never exceeds the budget.  Scenes rendered in a spawned process pool."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from paper_2203_02300_gb300 import scenes
    with ProcessPoolExecutor(8, mp_context=mp.get_context("spawn")) as ex:
        sc = list(ex.map(scenes.config_scene, [5] * 8, range(8)))
    pairs = [(torch.from_numpy(s.left).to(dev), torch.from_numpy(s.right).to(dev), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device=dev)) for s in sc]
    units = sum(s.W * s.H * s.D for s in sc)
    from paper_2203_02300_gb300 import tune
    with binding.Stereo(dev.index or 0, budget_bytes=budget) as h:
        t = _timed(torch, dev, flush, lambda: h.match_batch(pairs), reps)
        h.stream_status()
        alloc, groups = h.workspace_allocated(), h.batch_groups()
        # the blocks of the two 1-D passes from the autotuner (passes of 32
        # disparities, as the budget admits them)
        tile = tune.tune_shape(h, 1920, 1080, 256, device=dev.index or 0, max_slice_bytes=8 * 1920 * 1080 * 32)
        tuned = [p + (tile,) for p in pairs]
        t_tuned = _timed(torch, dev, flush, lambda: h.match_batch(tuned), reps)
        h.stream_status()
    return {"pairs": 8, "size": "1920x1080 D=256", "evals": units, "budget_bytes": budget,
            "one_volume_bytes": 1920 * 1080 * 256 * 4, "workspace_allocated_bytes": alloc,
            "admission_groups": groups, "ms": t, "evals_per_s": units / (t * 1e-3),
            "tuned_tile_d_h_v": list(tile), "tuned_ms": t_tuned, "tuned_evals_per_s": units / (t_tuned * 1e-3)}


def serve_config4_native(torch, binding, st, device: int, time_scale: float = 1.0, frames=None, tiles=None,
                         priorities=None):
    """Config 4 through the library's native serving runtime (dco_server_*:
    scheduler and completion threads in C++, maps copied straight into
    pinned output buffers); the same replay and comparison as serve_config4."""
    import numpy as np
    from paper_2203_02300_gb300 import scenes
    from paper_2203_02300_gb300.serve import run_config4_native
    clocks = Clocks(device if torch.cuda.device_count() > 1 else 0)
    clocks.start()
    stats, _, frames = run_config4_native(frames_per_stream=300, rate_hz=30.0, device=device, time_scale=time_scale,
                                          frames=frames, tiles=tiles,
                                          server_kw={"priorities": priorities} if priorities else None)
    stats = dict(stats, clocks=clocks.stop())
    stats["per_stream"] = {f"{W}x{H} D={D} (stream {k})": v for (W, H, D), (k, v) in
                           zip(scenes.STREAMS_CONFIG4, sorted(stats.get("per_stream", {}).items()))}
    return {"streams": [f"{W}x{H} D={D}" for W, H, D in scenes.STREAMS_CONFIG4],
            "frames_per_stream": 300, "unique_frames_per_stream": len(frames[0]), "rate_hz": 30 * time_scale,
            "tiles_d_h_v": [list(t) for t in tiles] if tiles else None,
            "latency_critical_streams": priorities or "none", **stats}


def serve_config4(torch, binding, st, device: int, time_scale: float = 1.0, frames=None, tiles=None):
    """4 camera streams, 300 frames each (cycled from 16 rendered ones per
    stream, planes moving 0-3 px per frame), Poisson arrivals at 30 Hz (real
    time): continuous batching over two lanes; p50/p99 from arrival to map on
    the host and where it goes (queue, device, host), against one plain
    synchronous call per frame size."""
    import numpy as np
    from paper_2203_02300_gb300 import scenes
    from paper_2203_02300_gb300.serve import run_config4
    stats, outs, frames = run_config4(frames_per_stream=300, rate_hz=30.0, device=device,
                                      time_scale=time_scale, frames=frames, server_kw={"tiles": tiles})
    plain = {}
    for i, (W, H, D) in enumerate(scenes.STREAMS_CONFIG4):
        l, r = frames[i][0]
        outh = np.empty((H, W), np.int16)
        p = binding.Tile.of(tiles[i] if tiles else None).apply(binding.Params.default())
        for _ in range(3):
            st.match_host(l.numpy(), r.numpy(), D, p, out=outh)
        ts = []
        for _ in range(20):
            t0 = time.perf_counter()
            st.match_host(l.numpy(), r.numpy(), D, p, out=outh)
            ts.append((time.perf_counter() - t0) * 1e3)
        plain[f"{W}x{H} D={D}"] = {"p50_ms": statistics.median(ts), "p99_ms": max(ts)}
        assert np.array_equal(outh, outs[(i, 0)]), "served map differs from the plain call"
    stats = dict(stats)
    stats["per_stream"] = {f"{W}x{H} D={D} (stream {k})": v for (W, H, D), (k, v) in
                           zip(scenes.STREAMS_CONFIG4, sorted(stats.get("per_stream", {}).items()))}
    return {"streams": [f"{W}x{H} D={D}" for W, H, D in scenes.STREAMS_CONFIG4],
            "frames_per_stream": 300, "unique_frames_per_stream": len(frames[0]), "rate_hz": 30 * time_scale,
            "tiles_d_h_v": [list(t) for t in tiles] if tiles else None, **stats, "plain_single_call": plain}


def serve_saturation(torch, device: int, frames, tiles, seconds: float = 3.0, native: bool = True):
    """Closed loop: every stream keeps its three slots busy for `seconds`;
    the serving throughput ceiling and the latency at that load."""
    from paper_2203_02300_gb300.serve import run_saturation, run_saturation_native
    if native:
        st = run_saturation_native(seconds, device=device, frames=frames, tiles=tiles)
    else:
        st = run_saturation(seconds, device=device, frames=frames, server_kw={"tiles": tiles})
    return {"seconds": seconds, "slots_per_stream": 3, "tiles_d_h_v": [list(t) for t in tiles] if tiles else None,
            **st}


# ------------------------------------------------------- oracle timing
def oracle_rate(scene, budget_s: float, rows_per_sample: int = 0):
    """The FP64 oracle as it stands, on all host cores, on row bands of the
    workload until about budget_s of CPU work; evals/s in the metric's unit."""
    from oracle import oracle as O
    cores = len(os.sched_getaffinity(0))
    O.set_threads(cores)
    rows = rows_per_sample or H
    done_units, t_used, y0, n = 0, 0.0, 0, 0
    while t_used < budget_s and n < 64:
        y1 = min(H, y0 + rows)
        t0 = time.perf_counter()
        O.match(scene.left, scene.right, D, rows=(y0, y1))
        t_used += time.perf_counter() - t0
        done_units += W * (y1 - y0) * D
        y0 = 0 if y1 >= H else y1
        n += 1
    # the same oracle on one core, one whole frame (a few seconds; a row band
    # would also compute its aggregation halo, which the units do not count)
    O.set_threads(1)
    t0 = time.perf_counter()
    O.match(scene.left, scene.right, D)
    t1 = time.perf_counter() - t0
    O.set_threads(cores)
    return {"value": done_units / t_used, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} oracle runs of {rows} rows x 640 cols x D=64 (both views + LR), "
                      f"{t_used:.1f} s of host time, FP64 C with OpenMP over rows",
            "single_core": {"value": W * H * D / t1, "unit": UNIT, "cores": 1,
                            "sample": f"one whole frame ({t1:.1f} s)"}}


def reference_arm(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from oracle import build as obuild
    from oracle import oracle as O
    from paper_2203_02300_gb300 import scenes
    obuild.build()
    s = scenes.config_scene(2)
    cores = len(os.sched_getaffinity(0))
    O.set_threads(cores)
    # one whole frame per step (about 0.15 s on 16 cores): a band would also
    # compute its aggregation halo, which the metric's units do not count
    rows = H
    for k in range(args.warmup):
        O.match(s.left, s.right, D)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        O.match(s.left, s.right, D)
        times.append(time.perf_counter() - t0)
    units = W * rows * D * args.steps
    value = units / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded plane scene)",
            "config": dict(CONFIG, sample_rows_per_step=rows),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "the whole 640x480 D=64 pair per step (both views + LR), FP64 C with "
                                       "OpenMP over rows"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
    else:
        own_arm(args)


if __name__ == "__main__":
    main()
