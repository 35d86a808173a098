"""Batched path (config 3: 32 pairs of uneven W x H x D in one pass of the
pipeline, one launch per stage) and its CUDA-graph replay.

The batched kernels run the same per-pair code as the single-pair path, so a
pair's disparity map must be bit-identical alone and inside a batch; a few
pairs are also checked against the oracle under the parity rule.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_02300_gb300 import scenes
from tests import parity

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def config3():
    return scenes.batch_config3(32)


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _single(env, s, params=None):
    torch, binding, st = env
    return st.match(_dev(torch, s.left), _dev(torch, s.right), s.D, params).cpu().numpy()


def test_config3_batch_equals_single(env, config3):
    torch, binding, st = env
    pairs = []
    for s in config3:
        L, R = _dev(torch, s.left), _dev(torch, s.right)
        pairs.append((L, R, s.D, torch.full((s.H, s.W), -9, dtype=torch.int16, device="cuda")))
    st.match_batch(pairs)
    torch.cuda.synchronize()
    st.sync_status()
    sizes = set()
    for s, (_, _, _, out) in zip(config3, pairs):
        sizes.add((s.W, s.H, s.D))
        assert np.array_equal(out.cpu().numpy(), _single(env, s)), (s.W, s.H, s.D)
    assert len(sizes) >= 3   # the batch really is uneven


def test_config3_batch_parity_full_frames(env, config3):
    # every distinct shape once (320x240 to 1280x720, D 32-128), whole frames
    # against the FP64 oracle
    torch, binding, st = env
    seen = {}
    for s in config3:
        seen.setdefault((s.W, s.H, s.D), s)
    pairs = []
    for s in seen.values():
        pairs.append((_dev(torch, s.left), _dev(torch, s.right), s.D,
                      torch.empty((s.H, s.W), dtype=torch.int16, device="cuda")))
    st.match_batch(pairs)
    torch.cuda.synchronize()
    tl, tr, tf = (parity.Tally(f"config 3 {v}") for v in ("left disparity", "right disparity", "final map"))
    for s, (L, R, _, out) in zip(seen.values(), pairs):
        got = out.cpu().numpy()
        fo, dl, dr, cl, cr = (t.cpu().numpy() for t in st.match_views(L, R, s.D))
        assert np.array_equal(got, fo)
        for rows in ((0, s.H),):
            ref = O.match(s.left, s.right, s.D, rows=rows, quantized=True)
            sl = slice(*rows)
            what = f"config 3 pair {s.W}x{s.H} D={s.D} full frame"
            parity.check_disparity(dl[sl], ref.disp_l, ref.best_l, ref.second_l, what + " left disparity",
                                   ref.qdisp_l, tally=tl)
            parity.check_disparity(dr[sl], ref.disp_r, ref.best_r, ref.second_r, what + " right disparity",
                                   ref.qdisp_r, tally=tr)
            parity.check_cost(cl[sl], ref.best_l, dl[sl], ref.disp_l, what + " left cost")
            parity.check_cost(cr[sl], ref.best_r, dr[sl], ref.disp_r, what + " right cost")
            parity.check_final(got[sl], ref, what + " final map (batch)", tally=tf)
    for t in (tl, tr, tf):
        t.close()


def test_more_pairs_than_one_launch_holds(env):
    # 70 small pairs: two launch groups per stage (64 + 6)
    torch, binding, st = env
    ss = [scenes.plane_scene(72 + (i % 5) * 8, 40 + (i % 3) * 8, 16 + (i % 2) * 8, 3,
                             seed=scenes.seed_for(3, 500 + i), drange=(1, 14)) for i in range(70)]
    pairs = [(_dev(torch, s.left), _dev(torch, s.right), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device="cuda")) for s in ss]
    st.match_batch(pairs)
    torch.cuda.synchronize()
    for s, (_, _, _, out) in zip(ss, pairs):
        assert np.array_equal(out.cpu().numpy(), _single(env, s))


def test_batch_with_several_passes(env, config3):
    torch, binding, st = env
    p = binding.Params.default(d_chunk=32)
    sub = config3[:8]
    pairs = [(_dev(torch, s.left), _dev(torch, s.right), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device="cuda")) for s in sub]
    st.match_batch(pairs, p)
    torch.cuda.synchronize()
    for s, (_, _, _, out) in zip(sub, pairs):
        assert np.array_equal(out.cpu().numpy(), _single(env, s))


def test_graph_replay_matches_direct_calls(env, config3):
    torch, binding, st = env
    from paper_2203_02300_gb300.batch import BatchGraph
    sub = config3[:6]
    g = BatchGraph(binding.Stereo(0), [(s.W, s.H, s.D) for s in sub])
    # second set: same shapes, different scenes, so a replay that ignored its
    # new inputs would fail
    other = [scenes.plane_scene(s.W, s.H, s.D, 5, seed=scenes.seed_for(3, 900 + i), drange=(2, s.D - 2),
                                noise_sigma=2.0) for i, s in enumerate(sub)]
    for batch in (sub, other, sub):
        outs = g([_dev(torch, s.left) for s in batch], [_dev(torch, s.right) for s in batch])
        torch.cuda.synchronize()
        for s, out in zip(batch, outs):
            assert np.array_equal(out.cpu().numpy(), _single(env, s))


def test_empty_and_invalid_batches(env):
    torch, binding, st = env
    st.match_batch([])
    L = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    out = torch.empty((8, 8), dtype=torch.int16, device="cuda")
    with pytest.raises(binding.DcoError) as e:
        st.match_batch([(L, L, 9, out)])   # D > W
    assert e.value.code == binding.DCO_EINVAL


def test_handles_never_lower_each_others_kernel_limits(env):
    # a wide pair needs more dynamic shared memory than a medium one; a second
    # handle running the medium pair must not lower the first handle's limit
    torch, binding, st = env
    a, b = binding.Stereo(0), binding.Stereo(0)
    wide = scenes.plane_scene(960, 96, 64, 4, seed=scenes.seed_for(3, 77), drange=(2, 60))
    mid = scenes.plane_scene(400, 96, 32, 4, seed=scenes.seed_for(3, 78), drange=(2, 30))
    r1 = a.match(_dev(torch, wide.left), _dev(torch, wide.right), wide.D).cpu().numpy()
    b.match(_dev(torch, mid.left), _dev(torch, mid.right), mid.D)
    r2 = a.match(_dev(torch, wide.left), _dev(torch, wide.right), wide.D).cpu().numpy()
    assert np.array_equal(r1, r2)
    a.close()
    b.close()


def test_batch_with_smoothing_equals_single(env, config3):
    torch, binding, st = env
    p = binding.Params.default(smooth_arms=1)
    sub = config3[:6]
    pairs = [(_dev(torch, s.left), _dev(torch, s.right), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device="cuda")) for s in sub]
    st.match_batch(pairs, p)
    torch.cuda.synchronize()
    for s, (_, _, _, out) in zip(sub, pairs):
        assert np.array_equal(out.cpu().numpy(), _single(env, s, p))


def test_batch_vh_order_equals_single(env, config3):
    # the other aggregation order: batched k_vcost / k_vagg row launches
    torch, binding, st = env
    p = binding.Params.default(agg_order=1)
    sub = config3[:8]
    pairs = [(_dev(torch, s.left), _dev(torch, s.right), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device="cuda")) for s in sub]
    st.match_batch(pairs, p)
    torch.cuda.synchronize()
    for s, (_, _, _, out) in zip(sub, pairs):
        assert np.array_equal(out.cpu().numpy(), _single(env, s, p))


def test_batch_with_per_pair_pass_widths(env, config3):
    # dco_pair_desc.d_chunk: each pair its own pass width (as the autotuner
    # picks per shape); results equal the pair alone, bit for bit
    torch, binding, st = env
    sub = config3[:8]
    widths = [32, 0, 64, 96, 0, 32, 128, 64]
    pairs = [(_dev(torch, s.left), _dev(torch, s.right), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device="cuda"), w) for s, w in zip(sub, widths)]
    st.match_batch(pairs)
    torch.cuda.synchronize()
    for s, pr in zip(sub, pairs):
        assert np.array_equal(pr[3].cpu().numpy(), _single(env, s))


def test_tuner_picks_a_candidate_and_caches_it(env, tmp_path, monkeypatch):
    torch, binding, st = env
    from paper_2203_02300_gb300 import tune
    monkeypatch.setenv("DCO_TUNE_CACHE", str(tmp_path / "tiles.json"))
    W, H, D = 320, 240, 96
    won = tune.tune_shape(st, W, H, D, reps=2)
    assert won.d_chunk in tune.candidates(W, H, D)
    assert won.h_chunk in tune.first_pass_candidates(W) and won.v_chunk in tune.second_pass_candidates(H)
    assert tune.lookup(W, H, D, torch.cuda.get_device_name(0)) == won
    assert tune.tune_batch(st, [(W, H, D), (W, H, D)]) == [won, won]
    # the tuned tile changes the speed, not the maps
    s = scenes.plane_scene(W, H, D, 4, seed=scenes.seed_for(3, 90), drange=(2, 90))
    l, r = _dev(torch, s.left), _dev(torch, s.right)
    assert torch.equal(st.match(l, r, D, won.apply(binding.Params.default())), st.match(l, r, D))


def test_batch_with_per_pair_tiles(env, config3):
    # dco_pair_desc h_chunk / v_chunk: each pair its own blocks of the two
    # 1-D passes; results equal the pair alone with automatic tiles
    torch, binding, st = env
    sub = config3[:8]
    tiles = [binding.Tile(0, 64, 0), binding.Tile(32, 0, 96), binding.Tile(0, 160, 120), binding.Tile(64, 96, 64),
             binding.Tile(), binding.Tile(0, 128, 200), binding.Tile(96, 320, 32), binding.Tile(0, 0, 50)]
    pairs = [(_dev(torch, s.left), _dev(torch, s.right), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device="cuda"), t) for s, t in zip(sub, tiles)]
    st.match_batch(pairs)
    torch.cuda.synchronize()
    for s, pr in zip(sub, pairs):
        assert np.array_equal(pr[3].cpu().numpy(), _single(env, s))
