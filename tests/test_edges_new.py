"""Edge cases of the Eq. 4 vote, the quarter-size depth, the smoothed arms and
the densification: single pixels, single rows and columns, D = 1, the
smallest valid sizes.  Integer results are compared bit for bit with the
oracle."""
import numpy as np
import pytest

from oracle import densify as DN
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


@pytest.mark.parametrize("W,H,D", [(1, 1, 1), (1, 9, 1), (9, 1, 3), (2, 2, 2), (40, 1, 8), (1, 40, 1)])
def test_vote_tiny(env, W, H, D):
    torch, binding, st = env
    rng = np.random.default_rng(W * 31 + H)
    img = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    d = rng.integers(-1, D, (H, W)).astype(np.int16)
    for smooth in (0, 1):
        p = binding.Params.default(vote_iters=2, smooth_arms=smooth)
        got = st.vote(_dev(torch, img), _dev(torch, d), D, p).cpu().numpy()
        assert np.array_equal(got, O.vote(d, O.arms(img, O.Params(smooth_arms=smooth)), D, 2)), (W, H, D, smooth)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 7), (7, 1), (2, 3)])
def test_smoothed_arms_tiny(env, W, H):
    torch, binding, st = env
    img = np.random.default_rng(W + 10 * H).integers(0, 256, (H, W, 3), dtype=np.uint8)
    got = st.arms(_dev(torch, img), binding.Params.default(smooth_arms=1)).cpu().numpy()
    assert np.array_equal(got, O.arms(img, O.Params(smooth_arms=1)))


@pytest.mark.parametrize("W,H,D", [(2, 2, 1), (3, 3, 1), (5, 2, 2), (2, 9, 1)])
def test_depth_smallest_sizes(env, W, H, D):
    torch, binding, st = env
    rng = np.random.default_rng(W * H)
    L = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    R = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    dh = torch.empty((H // 2, W // 2), dtype=torch.int16, device="cuda")
    z = st.depth(_dev(torch, L), _dev(torch, R), D, 500.0, 0.1, disp_half=dh).cpu().numpy()
    assert np.array_equal(st.downscale(_dev(torch, L)).cpu().numpy(), O.downscale(L))
    want = O.depth(dh.cpu().numpy(), W, H, 500.0, 0.1)
    assert np.allclose(z, want, rtol=1e-6, atol=0) and (z[want == 0] == 0).all()


@pytest.mark.parametrize("H,W", [(1, 1), (1, 12), (12, 1), (2, 2)])
def test_densify_tiny(env, H, W):
    torch, binding, st = env
    rng = np.random.default_rng(H * 7 + W)
    ds = np.where(rng.random((H, W)) < 0.5, rng.uniform(1, 4, (H, W)), 0.0).astype(np.float32)
    ds.flat[0] = 2.0
    z = np.zeros((H, W), np.float32)
    got = st.densify(_dev(torch, ds), None, _dev(torch, z), _dev(torch, z), None,
                     binding.DenseParams.default(tol=1e-6)).cpu().numpy()
    want = DN.densify(ds.astype(np.float64), np.zeros((H, W), np.uint8), z, z)
    assert np.allclose(got, want, rtol=1e-4, atol=1e-6)


def test_densify_without_any_data_is_all_missing(env):
    torch, binding, st = env
    z = np.zeros((5, 7), np.float32)
    got = st.densify(_dev(torch, z), None, _dev(torch, z), _dev(torch, z)).cpu().numpy()
    assert (got == 0).all()
    assert st.densify_stats()[0] == 0
