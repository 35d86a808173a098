"""Serving loop (config 4 pattern): several camera streams of different
sizes, Poisson arrivals, continuous batching over two lanes with memory-based
admission.  Every frame's map must equal the same frame matched alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(160, 120, 16), (200, 150, 24), (320, 240, 32)]


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_02300_gb300 import binding
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device")
    st = binding.Stereo(0)
    yield torch, binding, st
    st.close()


def _alone(env, frames):
    torch, binding, st = env
    res = {}
    for i, fr in enumerate(frames):
        for k, (l, r) in enumerate(fr):
            D = SHAPES[i][2]
            res[(i, k)] = st.match(l.cuda(), r.cuda(), D).cpu().numpy()
    return res


def test_served_results_equal_alone(env):
    from paper_2203_02300_gb300.serve import run_config4
    stats, outs, frames = run_config4(frames_per_stream=24, rate_hz=400.0, unique_frames=4, shapes=SHAPES)
    alone = _alone(env, frames)
    for (i, k), got in outs.items():
        assert np.array_equal(got, alone[(i, k % 4)]), (i, k)
    assert stats["frames"] == 24 * len(SHAPES)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_burst_is_batched_and_memory_admission_holds(env):
    torch, binding, st = env
    from paper_2203_02300_gb300 import scenes
    from paper_2203_02300_gb300.serve import Server
    frames = [[(torch.from_numpy(s.left).pin_memory(), torch.from_numpy(s.right).pin_memory())
               for s in [scenes.StreamScene(i, W, H, D).frame(t) for t in range(2)]]
              for i, (W, H, D) in enumerate(SHAPES)]
    ws = [binding.Stereo.workspace_bytes(W, H, D) for (W, H, D) in SHAPES]
    budget = 2 * (ws[2] + ws[1])          # per lane: the largest and the middle stream at most
    srv = Server(SHAPES, budget_bytes=budget, lanes=2, slots_per_stream=2, max_batch=8)
    futs = []
    for rep in range(3):
        for i in range(len(SHAPES)):
            for k in range(2):
                futs.append(((i, k), srv.submit(i, *frames[i][k])))
    outs = [(key, f.result(timeout=60)) for key, f in futs]
    srv.close()
    stats = srv.stats()
    alone = _alone(env, frames)
    for key, got in outs:
        assert np.array_equal(got, alone[key])
    assert stats["mean_batch"] > 1.0          # a burst is served in batches
    # no batch needed more workspace than a lane's share of the budget, and
    # the budget really limited the batches (all 18 frames would need more)
    assert 0 < srv.max_batch_bytes <= srv.lane_budget == budget // 2
    assert 3 * 2 * sum(ws) > srv.lane_budget


def test_config4_full_size_streams_against_the_oracle(env):
    # the four config 4 streams at their real sizes (640x480 D=64, 960x540
    # D=96, 1280x720 D=128 twice), three distinct frames each (planes moving
    # between frames), Poisson arrivals at 30 Hz: every served map equals the
    # frame matched alone, and the first frame of every stream passes the
    # parity rule against the FP64 oracle on the whole frame
    from oracle import oracle as O
    from paper_2203_02300_gb300 import scenes
    from paper_2203_02300_gb300.serve import run_config4
    from tests import parity
    torch, binding, st = env
    stats, outs, frames = run_config4(frames_per_stream=3, rate_hz=30.0, unique_frames=3)
    assert stats["frames"] == 3 * len(scenes.STREAMS_CONFIG4)
    for (i, k), got in outs.items():
        W, H, D = scenes.STREAMS_CONFIG4[i]
        l, r = frames[i][k]
        assert np.array_equal(got, st.match(l.cuda(), r.cuda(), D).cpu().numpy()), (i, k)
        if k == 0:
            ref = O.match(l.numpy(), r.numpy(), D)
            parity.check_final(got, ref, f"config 4 stream {i} ({W}x{H} D={D}) frame 0 final map")


def test_native_runtime_results_equal_alone(env):
    # the library's serving runtime (dco_server_*): frames of three streams at
    # 400 Hz each, every map equal to the frame matched alone
    from paper_2203_02300_gb300.serve import run_config4_native
    stats, outs, frames = run_config4_native(frames_per_stream=16, rate_hz=400.0, unique_frames=4, shapes=SHAPES,
                                             keep_outputs=True)
    alone = _alone(env, frames)
    for (i, k), got in outs.items():
        assert np.array_equal(got, alone[(i, k % 4)]), (i, k)
    assert stats["frames"] == 16 * len(SHAPES)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["latency_parts"]["device"]["p50_ms"] > 0


def test_native_runtime_batches_a_burst_within_the_budget(env):
    torch, binding, st = env
    from paper_2203_02300_gb300 import scenes
    frames = [[(torch.from_numpy(s.left).pin_memory().numpy(), torch.from_numpy(s.right).pin_memory().numpy())
               for s in [scenes.StreamScene(i, W, H, D).frame(t) for t in range(2)]]
              for i, (W, H, D) in enumerate(SHAPES)]
    ws = [binding.Stereo.workspace_bytes(W, H, D) for (W, H, D) in SHAPES]
    budget = 2 * (ws[2] + ws[1])
    # every output buffer exists before the first submit, so the 18 requests
    # arrive within microseconds; one lane: while it runs the first frame the
    # others queue up and are admitted in batches
    outs = [((i, k), torch.full((H, W), -9, dtype=torch.int16).pin_memory().numpy())
            for rep in range(3) for i, (W, H, D) in enumerate(SHAPES) for k in range(2)]
    tickets = []
    with binding.NativeServer(SHAPES, budget_bytes=budget, lanes=1, slots_per_stream=2, max_batch=8) as srv:
        for (i, k), o in outs:
            tickets.append(srv.submit(i, frames[i][k][0], frames[i][k][1], o))
        for t in tickets:
            srv.wait(t, timeout_ms=60000)
        cnt = srv.counters()
    alone = {}
    for i, (W, H, D) in enumerate(SHAPES):
        for k in range(2):
            alone[(i, k)] = st.match(torch.from_numpy(frames[i][k][0]).cuda(), torch.from_numpy(frames[i][k][1]).cuda(),
                                     D).cpu().numpy()
    for key, got in outs:
        assert np.array_equal(got, alone[key])
    assert cnt["frames"] == 18 and cnt["frames"] / cnt["batches"] > 1.0   # a burst is served in batches
    assert 0 < cnt["max_batch_bytes"] <= cnt["lane_budget"] == budget


def test_native_runtime_rejects_bad_requests(env):
    torch, binding, st = env
    import pytest as _pt
    with binding.NativeServer(SHAPES[:1]) as srv:
        W, H, _ = SHAPES[0]
        l = np.zeros((H, W, 3), np.uint8)
        o = np.zeros((H, W), np.int16)
        with _pt.raises(binding.DcoError) as e:
            binding._check(binding.lib().dco_server_submit(srv._s, 5, l.ctypes.data, l.ctypes.data, o.ctypes.data,
                                                           binding.ctypes.byref(binding.ctypes.c_ulonglong())), None)
        assert e.value.code == binding.DCO_EINVAL
        with _pt.raises(binding.DcoError) as e:
            srv.wait(12345)
        assert e.value.code == binding.DCO_EINVAL
    with _pt.raises(binding.DcoError) as e:   # a lane's share cannot hold one frame
        binding.NativeServer(SHAPES, budget_bytes=1000)
    assert e.value.code == binding.DCO_EBUDGET
    for bad in (dict(priorities=[2] + [0] * (len(SHAPES) - 1)), dict(tiles=[(0, 16, 0)] * len(SHAPES))):
        with _pt.raises(binding.DcoError) as e:
            binding.NativeServer(SHAPES, **bad)
        assert e.value.code == binding.DCO_EINVAL


def test_native_runtime_with_latency_critical_streams_equals_alone(env):
    # the smaller streams marked latency-critical: admitted first, batched
    # only with each other, run on high-priority CUDA streams; every map
    # still equals the frame matched alone
    from paper_2203_02300_gb300.serve import run_config4_native
    stats, outs, frames = run_config4_native(frames_per_stream=16, rate_hz=400.0, unique_frames=4, shapes=SHAPES,
                                             keep_outputs=True, server_kw={"priorities": "smaller"})
    alone = _alone(env, frames)
    for (i, k), got in outs.items():
        assert np.array_equal(got, alone[(i, k % 4)]), (i, k)
    assert stats["frames"] == 16 * len(SHAPES)


def test_native_runtime_pageable_and_pinned_buffers(env):
    # pinned buffers are read and written in place by the kernels, pageable
    # ones go through the stream's device slots; both give the map matched
    # alone, also mixed within one stream
    torch, binding, st = env
    from paper_2203_02300_gb300 import scenes
    W, H, D = SHAPES[1]
    sc = [scenes.StreamScene(1, W, H, D).frame(t) for t in range(4)]
    alone = [st.match(torch.from_numpy(s.left).cuda(), torch.from_numpy(s.right).cuda(), D).cpu().numpy() for s in sc]
    jobs = []
    with binding.NativeServer([(W, H, D)], lanes=2, slots_per_stream=2) as srv:
        for k, s in enumerate(sc * 3):
            pinned = k % 2 == 0
            if pinned:
                l = torch.from_numpy(s.left).pin_memory().numpy()
                r = torch.from_numpy(s.right).pin_memory().numpy()
                o = torch.full((H, W), -9, dtype=torch.int16).pin_memory().numpy()
            else:
                l, r, o = s.left.copy(), s.right.copy(), np.full((H, W), -9, np.int16)
            jobs.append((k % 4, o, srv.submit(0, l, r, o)))
        for k, o, t in jobs:
            srv.wait(t, timeout_ms=60000)
    for k, o, t in jobs:
        assert np.array_equal(o, alone[k]), k
