"""Failure handling and repeatability of the C ABI, with no GPU fault.

- An allocation the device cannot satisfy is reported as DCO_ENOMEM, and the
  handle stays usable: the next calls allocate what they need and their
  launch checks are not confused by the failed allocation.
- A map does not depend on what the workspace held before: the same pair
  gives bit-identical maps on a fresh handle and after other pairs (other
  sizes, other disparity ranges and pass widths) have used the workspace.
"""
import numpy as np
import pytest

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


def test_allocation_failure_is_reported_and_recoverable(env):
    torch, binding, st = env
    s = scenes.config_scene(1)
    L, R = _dev(torch, s.left), _dev(torch, s.right)
    want = st.match(L, R, s.D).cpu().numpy()
    # one pass over 256 disparities of a 16384 x 16384 pair: about 550 GB of
    # slices, more than the device holds
    p = binding.Params.default(d_chunk=256)
    assert binding.Stereo.workspace_bytes(16384, 16384, 256, p) > torch.cuda.get_device_properties(0).total_memory
    with binding.Stereo(0) as h:
        for _ in range(2):
            with pytest.raises(binding.DcoError) as e:
                h.reserve(16384, 16384, 256, p)
            assert e.value.code == binding.DCO_ENOMEM
        # the handle still works, and its launches report no stale error
        got = h.match(L, R, s.D).cpu().numpy()
        torch.cuda.synchronize()
        h.sync_status()
    assert np.array_equal(got, want)
    # the shared handle is unaffected as well
    assert np.array_equal(st.match(L, R, s.D).cpu().numpy(), want)


def test_maps_do_not_depend_on_the_workspace_history(env):
    torch, binding, _ = env
    a = scenes.config_scene(1)                                                   # 320x240, D=32
    b = scenes.plane_scene(333, 211, 45, 6, seed=scenes.seed_for(9, 1), drange=(2, 40), noise_sigma=2.0,
                           texture="mixed")
    c = scenes.plane_scene(640, 120, 96, 6, seed=scenes.seed_for(9, 5), drange=(2, 90), noise_sigma=2.0,
                           texture="mixed")
    pairs = [(a, None), (b, binding.Params.default(d_chunk=16)), (c, binding.Params.default(vote_iters=1)),
             (b, None)]

    def run(h, sc, p):
        out, dl, dr, cl, cr = h.match_views(_dev(torch, sc.left), _dev(torch, sc.right), sc.D, p)
        torch.cuda.synchronize()
        return [t.cpu().numpy() for t in (out, dl, dr, cl, cr)]

    fresh = []
    for sc, p in pairs:
        with binding.Stereo(0) as h:
            fresh.append(run(h, sc, p))
    with binding.Stereo(0) as h:   # one handle, every pair twice, in two orders
        for order in (range(len(pairs)), reversed(range(len(pairs)))):
            for k in order:
                got = run(h, *pairs[k])
                for g, w in zip(got, fresh[k]):
                    assert np.array_equal(g, w)
        h.sync_status()


def test_lost_tile_copies_time_out_and_the_context_stays_usable(env):
    # failure test flag: the V pass arms each tile's mbarrier but issues no
    # copy, so every bounded wait runs out with nothing in flight; the kernel
    # sets bit 0 of the status word and returns (no trap, no hang)
    torch, binding, _ = env
    s = scenes.plane_scene(96, 64, 16, 3, seed=scenes.seed_for(9, 20), drange=(2, 13))
    L, R = _dev(torch, s.left), _dev(torch, s.right)
    with binding.Stereo(0) as h:
        want = h.match(L, R, s.D).cpu().numpy()
        h.stream_status()
        h.set_test_flags(binding.DCO_TEST_LOSE_TILE_COPIES)
        h.match(L, R, s.D)
        with pytest.raises(binding.DcoError) as e:
            h.stream_status()
        assert e.value.code == binding.DCO_ETIMEOUT
        h.stream_status()   # the read cleared the word
        with pytest.raises(binding.DcoError):
            h.set_test_flags(2)
        h.set_test_flags(0)
        got = h.match(L, R, s.D).cpu().numpy()
        h.stream_status()
        torch.cuda.synchronize()
    assert np.array_equal(got, want)


def test_lost_grid_arrival_times_out_and_the_handle_stays_usable(env):
    # failure test flag: in the one-launch densification solve, block 0 never
    # arrives at the first grid barrier and every barrier waits only a few
    # polls, so all blocks give up and return (no trap, no hang); the call
    # reports DCO_ETIMEOUT and the same handle then solves normally
    torch, binding, _ = env
    rng = np.random.default_rng(12)
    H, W = 64, 96
    ds = np.where(rng.random((H, W)) < 0.2, rng.uniform(0.5, 5.0, (H, W)), 0.0).astype(np.float32)
    mi = rng.random((H, W)).astype(np.float32)
    d_ds, d_mi = _dev(torch, ds), _dev(torch, mi)
    p = binding.DenseParams.default(tol=1e-6)
    with binding.Stereo(0) as h:
        want = h.densify(d_ds, None, d_mi, d_mi, None, p).cpu().numpy()
        h.set_test_flags(binding.DCO_TEST_LOSE_GRID_ARRIVAL)
        with pytest.raises(binding.DcoError) as e:
            h.densify(d_ds, None, d_mi, d_mi, None, p)
        assert e.value.code == binding.DCO_ETIMEOUT
        h.set_test_flags(0)
        got = h.densify(d_ds, None, d_mi, d_mi, None, p).cpu().numpy()
        torch.cuda.synchronize()
    assert np.array_equal(got, want)


def test_stream_status_waits_for_its_own_stream(env):
    torch, binding, _ = env
    s = scenes.config_scene(1)
    L, R = _dev(torch, s.left), _dev(torch, s.right)
    side = torch.cuda.Stream()
    with binding.Stereo(0) as h:
        with torch.cuda.stream(side):
            out = h.match(L, R, s.D, stream=side)
            h.stream_status(side)   # returns once `side` has finished the match
        assert side.query()
        got = out.cpu().numpy()
    with binding.Stereo(0) as h:
        assert np.array_equal(got, h.match(L, R, s.D).cpu().numpy())
