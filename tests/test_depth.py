"""Quarter-size input and sparse depth (Sect. 4, 4.4) on the GPU against the
oracle: the downscale is integer work (bit-exact), the half-size map is the
matcher's own (bit-identical to matching the downscaled pair), the depth is
one FP32 division per pixel (relative error <= 2^-23 of FP64: tolerance
1e-6 relative, exact zeros where depth is missing)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_02300_gb300 import scenes

pytestmark = pytest.mark.gpu
F_PX, BASE = 700.0, 0.12


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


@pytest.mark.parametrize("W,H", [(2, 2), (64, 48), (161, 97), (1280, 720)])
def test_downscale_bit_exact(env, W, H):
    torch, binding, st = env
    rng = np.random.default_rng(W + H)
    img = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    assert np.array_equal(st.downscale(_dev(torch, img)).cpu().numpy(), O.downscale(img))


@pytest.mark.parametrize("W,H,D,vote", [(128, 96, 16, 0), (161, 97, 24, 1), (640, 480, 32, 0)])
def test_depth_equals_oracle_on_the_matchers_map(env, W, H, D, vote):
    torch, binding, st = env
    s = scenes.plane_scene(W, H, 2 * D, 6, seed=scenes.seed_for(2, 600 + W), drange=(2, 2 * D - 4))
    L, R = _dev(torch, s.left), _dev(torch, s.right)
    p = binding.Params.default(vote_iters=vote)
    dh = torch.empty((H // 2, W // 2), dtype=torch.int16, device="cuda")
    z = st.depth(L, R, D, F_PX, BASE, p, disp_half=dh).cpu().numpy()
    st.sync_status()
    dh = dh.cpu().numpy()
    # the half-size map is the matcher's own on the downscaled pair
    Lh, Rh = st.downscale(L), st.downscale(R)
    assert np.array_equal(dh, st.match(Lh, Rh, D, p).cpu().numpy())
    want = O.depth(dh, W, H, F_PX, BASE)
    miss = want == 0
    assert (z[miss] == 0).all()
    assert np.allclose(z[~miss], want[~miss], rtol=1e-6, atol=0)
    assert (~miss).mean() > 0.3


def test_depth_matches_the_oracle_path_under_the_parity_rule(env):
    # the whole chain against the oracle's own chain: downscale, match, depth
    torch, binding, st = env
    from tests import parity
    s = scenes.plane_scene(160, 120, 32, 5, seed=scenes.seed_for(2, 650), drange=(2, 28))
    dh = torch.empty((60, 80), dtype=torch.int16, device="cuda")
    st.depth(_dev(torch, s.left), _dev(torch, s.right), 16, F_PX, BASE, disp_half=dh)
    ref = O.match(O.downscale(s.left), O.downscale(s.right), 16, quantized=True)
    parity.check_final(dh.cpu().numpy(), ref, "half-size map")


def test_depth_recovers_a_plane(env):
    torch, binding, st = env
    d0 = 6
    s = scenes.plane_scene(256, 192, 32, 0, seed=31, drange=(2 * d0, 2 * d0))
    z = st.depth(_dev(torch, s.left), _dev(torch, s.right), 16, F_PX, BASE).cpu().numpy()
    interior = z[16:-16, 2 * (d0 + 16):-16]
    assert np.isclose(interior, F_PX * BASE / (2 * d0), rtol=1e-6).mean() > 0.95


def test_depth_rejects_bad_arguments(env):
    torch, binding, st = env
    L = torch.zeros((8, 8, 3), dtype=torch.uint8, device="cuda")
    for args in ((4, 0.0, 0.1), (4, 700.0, -1.0), (5, 700.0, 0.1)):   # f, B, D > W/2
        with pytest.raises(binding.DcoError) as e:
            st.depth(L, L, args[0], args[1], args[2])
        assert e.value.code == binding.DCO_EINVAL
    one = torch.zeros((1, 8, 3), dtype=torch.uint8, device="cuda")
    with pytest.raises(binding.DcoError):
        st.depth(one, one, 2, 700.0, 0.1)
