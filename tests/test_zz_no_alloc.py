"""The allocation-free entry point (dco_stereo_match_noalloc).

Some callers cannot allocate device memory (where cudaMalloc is forbidden or
the memory footprint must stay fixed after start-up).  For them the library
exports one entry point whose scratch lives in a static device array.  This
file checks, through the C ABI, that it returns the same disparity maps as
the regular entry point on two calls in a row (the second call must not be
affected by what the first left in the shared array), that the array's
status word reads clean after each call, and that sizes beyond the array
are rejected before any work.  It runs last so that a failure here
never hides the other tests, and passes in a fresh process or after them.
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


def _noalloc(env, left, right, D):
    torch, binding, st = env
    L = torch.from_numpy(left).cuda()
    R = torch.from_numpy(right).cuda()
    H, W, _ = left.shape
    out = torch.full((H, W), -7, dtype=torch.int16, device="cuda")
    rc = binding.lib().dco_stereo_match_noalloc(L.data_ptr(), R.data_ptr(), W, H, D, None, out.data_ptr(),
                                                torch.cuda.current_stream().cuda_stream)
    assert rc == binding.DCO_OK, binding.STATUS.get(rc, rc)
    ref = st.match(L, R, D)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ref.cpu().numpy()


def test_two_calls_match_the_regular_entry_point(env):
    a = scenes.config_scene(1)                                   # 320x240, D=32
    b = scenes.plane_scene(256, 200, 48, 6, seed=scenes.seed_for(1, 5), drange=(2, 44), noise_sigma=2.0)
    for s in (a, b):
        got, want = _noalloc(env, s.left, s.right, s.D)
        # same kernels on the same inputs: the consistency maps agree exactly
        # (tolerance of integer work); also within the oracle's parity rule
        assert np.array_equal(got, want)
        ref = O.match(s.left, s.right, s.D)
        parity.check_final(got, ref, "no-alloc")
        # the status word in the array reports no device-side failure (and
        # is cleared by the read)
        torch, binding, st = env
        assert binding.lib().dco_stereo_noalloc_status(torch.cuda.current_stream().cuda_stream) == binding.DCO_OK


def test_sizes_beyond_the_array_are_rejected(env):
    torch, binding, st = env
    big = torch.zeros((720, 1280, 3), dtype=torch.uint8, device="cuda")
    out = torch.full((720, 1280), -7, dtype=torch.int16, device="cuda")
    rc = binding.lib().dco_stereo_match_noalloc(big.data_ptr(), big.data_ptr(), 1280, 720, 64, None,
                                                out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == binding.DCO_EBUDGET
    torch.cuda.synchronize()
    assert (out == -7).all()   # nothing was enqueued
