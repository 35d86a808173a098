"""Eq. 4 parallax optimisation on the GPU against the oracle (bit-exact:
integer counts and an argmax with the smallest d on ties), on the same
input map and image (the arms are bit-exact already)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_02300_gb300 import scenes

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


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _noisy_map(rng, s, D, p_invalid=0.15, p_outlier=0.1):
    """Ground-truth disparities with outliers, invalid (-1) and out-of-range values."""
    d = np.clip(np.rint(s.disp), 0, D - 1).astype(np.int16)
    u = rng.random(d.shape)
    d[u < p_outlier] = rng.integers(0, D, int((u < p_outlier).sum()))
    d[(u >= p_outlier) & (u < p_outlier + p_invalid)] = -1
    d[rng.random(d.shape) < 0.01] = D + 3
    return d


@pytest.mark.parametrize("W,H,D,chunk,iters", [(96, 64, 16, 0, 1), (77, 53, 20, 0, 3), (200, 150, 48, 32, 2),
                                                 (130, 41, 64, 0, 1), (33, 200, 24, 0, 2)])
def test_vote_equals_oracle(env, W, H, D, chunk, iters):
    torch, binding, st = env
    rng = np.random.default_rng(W * H + D)
    s = scenes.plane_scene(W, H, D, 5, seed=scenes.seed_for(1, 300 + W), drange=(1, D - 2))
    d = _noisy_map(rng, s, D)
    p = binding.Params.default(d_chunk=chunk, vote_iters=iters)
    got = st.vote(_dev(torch, s.left), _dev(torch, d), D, p).cpu().numpy()
    st.sync_status()
    want = O.vote(d, O.arms(s.left), D, iters)
    assert np.array_equal(got, want)
    assert (got[(d < 0) | (d >= D)] == -1).all()


def test_vote_with_tiles_equals_oracle(env):
    # the vote's passes use the call's blocks of the two 1-D passes too
    torch, binding, st = env
    rng = np.random.default_rng(17)
    s = scenes.plane_scene(200, 150, 48, 5, seed=scenes.seed_for(1, 330), drange=(1, 46))
    d = _noisy_map(rng, s, 48)
    want = O.vote(d, O.arms(s.left), 48, 2)
    for h, v in ((64, 48), (32, 32), (128, 0), (0, 100)):
        p = binding.Params.default(vote_iters=2, h_chunk=h, v_chunk=v)
        got = st.vote(_dev(torch, s.left), _dev(torch, d), 48, p).cpu().numpy()
        st.sync_status()
        assert np.array_equal(got, want), (h, v)


def test_vote_removes_outliers(env):
    torch, binding, st = env
    rng = np.random.default_rng(7)
    s = scenes.plane_scene(160, 120, 32, 4, seed=scenes.seed_for(1, 310), drange=(2, 28))
    d = _noisy_map(rng, s, 32, p_invalid=0.0, p_outlier=0.2)
    got = st.vote(_dev(torch, s.left), _dev(torch, d), 32, binding.Params.default(vote_iters=2)).cpu().numpy()
    gt = np.clip(np.rint(s.disp), 0, 31)
    valid = (d >= 0) & (d < 32)
    assert (got[valid] == gt[valid]).mean() > (d[valid] == gt[valid]).mean() + 0.1


def test_vote_in_place_and_zero_rounds(env):
    torch, binding, st = env
    rng = np.random.default_rng(8)
    s = scenes.plane_scene(64, 48, 16, 3, seed=scenes.seed_for(1, 320), drange=(1, 14))
    d = _noisy_map(rng, s, 16)
    img = _dev(torch, s.left)
    t = _dev(torch, d)
    st.vote(img, t, 16, binding.Params.default(vote_iters=2), out=t)
    assert np.array_equal(t.cpu().numpy(), O.vote(d, O.arms(s.left), 16, 2))
    z = st.vote(img, _dev(torch, d), 16, binding.Params.default(vote_iters=0)).cpu().numpy()
    assert np.array_equal(z, d)


def test_match_with_vote_is_vote_of_the_checked_map(env):
    torch, binding, st = env
    s = scenes.config_scene(1)
    L, R = _dev(torch, s.left), _dev(torch, s.right)
    base = st.match(L, R, s.D, binding.Params.default()).cpu().numpy()
    for iters in (1, 2):
        got = st.match(L, R, s.D, binding.Params.default(vote_iters=iters)).cpu().numpy()
        assert np.array_equal(got, O.vote(base, O.arms(s.left), s.D, iters)), iters


def test_batch_with_vote_equals_single(env):
    torch, binding, st = env
    p = binding.Params.default(vote_iters=1)
    ss = [scenes.plane_scene(96 + 16 * i, 64 + 8 * i, 16 + 8 * (i % 2), 3, seed=scenes.seed_for(3, 700 + i),
                             drange=(1, 14)) for i in range(5)]
    pairs = [(_dev(torch, s.left), _dev(torch, s.right), s.D,
              torch.empty((s.H, s.W), dtype=torch.int16, device="cuda")) for s in ss]
    st.match_batch(pairs, p)
    torch.cuda.synchronize()
    for s, (l, r, D, out) in zip(ss, pairs):
        assert np.array_equal(out.cpu().numpy(), st.match(l, r, D, p).cpu().numpy())


def test_vote_full_size_config2(env):
    torch, binding, st = env
    s = scenes.config_scene(2)
    rng = np.random.default_rng(9)
    d = _noisy_map(rng, s, s.D)
    got = st.vote(_dev(torch, s.left), _dev(torch, d), s.D, binding.Params.default(vote_iters=1)).cpu().numpy()
    assert np.array_equal(got, O.vote(d, O.arms(s.left), s.D, 1))


def test_vote_rejects_bad_rounds(env):
    torch, binding, st = env
    img = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    d = torch.zeros((8, 8), dtype=torch.int16, device="cuda")
    with pytest.raises(binding.DcoError) as e:
        st.vote(img, d, 4, binding.Params.default(vote_iters=65))
    assert e.value.code == binding.DCO_EINVAL


def test_vote_over_smoothed_arms(env):
    torch, binding, st = env
    rng = np.random.default_rng(10)
    s = scenes.plane_scene(120, 90, 24, 5, seed=scenes.seed_for(1, 330), drange=(1, 22), noise_sigma=2.0)
    d = _noisy_map(rng, s, 24)
    p = binding.Params.default(vote_iters=2, smooth_arms=1)
    got = st.vote(_dev(torch, s.left), _dev(torch, d), 24, p).cpu().numpy()
    assert np.array_equal(got, O.vote(d, O.arms(s.left, O.Params(smooth_arms=1)), 24, 2))


@pytest.mark.parametrize("over", [dict(), dict(agg_order=1), dict(smooth_arms=1), dict(agg_order=1, smooth_arms=1)])
def test_whole_path_with_vote_equals_the_oracle_chain(env, over):
    # the path with two Eq. 4 rounds equals the oracle's vote (over the
    # order-0 regions of the possibly smoothed left arms) applied to the
    # GPU's checked map, and that map passes the parity rule against the
    # FP64 oracle; where it equals the FP64 map exactly, the whole chain is
    # the oracle's own
    torch, binding, st = env
    from tests import parity
    s = scenes.plane_scene(160, 96, 24, 4, seed=scenes.seed_for(2, 990), slanted=True, noise_sigma=2.0,
                           drange=(2, 21), texture="mixed")
    L, R = _dev(torch, s.left), _dev(torch, s.right)
    got = st.match(L, R, s.D, binding.Params.default(vote_iters=2, **over)).cpu().numpy()
    plain = st.match(L, R, s.D, binding.Params.default(**over)).cpu().numpy()
    op = O.Params(**over)
    ref = O.match(s.left, s.right, s.D, op)
    parity.check_final(plain, ref, f"vote chain {over} checked map")
    arm = O.arms(s.left, op)
    assert np.array_equal(got, O.vote(plain, arm, s.D, 2))
    if np.array_equal(plain, ref.disp):
        assert np.array_equal(got, O.vote(ref.disp, arm, s.D, 2))
