"""Depth densification (Sect. 6, Eqs. 13-20) on the GPU against the FP64
oracle (sparse direct solve of the same normal equations).  The GPU solve is
conjugate gradients in FP32 stopped at a relative residual `tol`; the tests
check (a) that residual, recomputed in FP64 with the oracle's own system,
(b) the solution against the direct solve, and (c) exact zeros where Eq. 20
leaves the depth undetermined."""
import numpy as np
import pytest

from oracle import densify as DN
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


def _dev(torch, a, dt=None):
    import torch as T
    return T.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _inputs(rng, H, W, frac=0.1, contour=True, pre=True):
    ds = np.where(rng.random((H, W)) < frac, rng.uniform(0.5, 5.0, (H, W)), 0.0).astype(np.float32)
    B = (rng.random((H, W)) < 0.1).astype(np.uint8) if contour else np.zeros((H, W), np.uint8)
    mf = rng.random((H, W)).astype(np.float32)
    mi = rng.random((H, W)).astype(np.float32)
    dp = np.where(rng.random((H, W)) < 0.2, rng.uniform(1, 3, (H, W)), 0.0).astype(np.float32) if pre else None
    return ds, B, mf, mi, dp


def _solve(env, ds, B, mf, mi, dp, **over):
    torch, binding, st = env
    p = binding.DenseParams.default(**over)
    out = st.densify(_dev(torch, ds), _dev(torch, B) if B is not None else None, _dev(torch, mf), _dev(torch, mi),
                     _dev(torch, dp) if dp is not None else None, p).cpu().numpy()
    st.sync_status()
    return out, st.densify_stats()


def _true_relres(x, ds, B, mf, mi, dp, p):
    A, b = DN.system(ds.astype(np.float64), B, mf, mi, None if dp is None else dp.astype(np.float64), p)
    r = b - A @ x.astype(np.float64).ravel()
    return np.linalg.norm(r) / np.linalg.norm(b)


# The attainable residual relative to ||b|| is bounded by the FP32 storage of
# x: about 2^-24 * |A x| per pixel against b, which is nonzero only where data
# exist, so sparser data need a larger tol (2 % data: ~5e-6 at best).
@pytest.mark.parametrize("solver", [0, 1])
@pytest.mark.parametrize("H,W,frac,tol", [(30, 40, 0.1, 1e-6), (61, 97, 0.3, 1e-6), (17, 230, 0.02, 2e-5)])
def test_densify_equals_the_direct_solve(env, H, W, frac, tol, solver):
    # solver 0: one cooperative launch for the solve; 1: two launches per iteration
    rng = np.random.default_rng(H * W)
    ds, B, mf, mi, dp = _inputs(rng, H, W, frac)
    x, (iters, rel) = _solve(env, ds, B, mf, mi, dp, tol=tol, max_iters=20000, solver=solver)
    p = DN.DenseParams()
    want = DN.densify(ds.astype(np.float64), B, mf, mi, dp.astype(np.float64), p)
    assert 0 < iters < 20000 and rel <= tol
    assert _true_relres(x, ds, B, mf, mi, dp, p) <= 2.5 * tol
    assert np.abs(x - want).max() <= 1e-3 * np.abs(want).max()
    assert (x[want == 0] == 0).all()


def test_densify_single_anchor_and_contour_split(env):
    z = np.zeros((9, 11), np.float32)
    ds = z.copy(); ds[4, 5] = 2.5
    x, _ = _solve(env, ds, None, z, z, None, tol=1e-7)
    assert np.allclose(x, 2.5, rtol=1e-5)
    ds = np.zeros((6, 10), np.float32); ds[2, 1] = 1.0; ds[3, 8] = 4.0
    B = np.zeros((6, 10), np.uint8); B[:, 5:] = 1
    x, _ = _solve(env, ds, B, np.zeros((6, 10), np.float32), np.zeros((6, 10), np.float32), None, tol=1e-7)
    assert np.allclose(x[:, :5], 1.0, rtol=1e-5) and np.allclose(x[:, 5:], 4.0, rtol=1e-5)


@pytest.mark.parametrize("solver", [0, 1])
def test_densify_without_smoothness_is_the_data(env, solver):
    rng = np.random.default_rng(3)
    ds, B, mf, mi, dp = _inputs(rng, 20, 30, 0.5)
    x, (iters, _) = _solve(env, ds, B, mf, mi, dp, lambda_s=0.0, tol=1e-7, solver=solver)
    ws, wt = (ds > 0) * 0.8, (dp > 0) * 0.02
    want = np.where(ws + wt > 0, (ws * ds + wt * dp) / np.where(ws + wt > 0, ws + wt, 1), 0.0)
    assert np.allclose(x, want, rtol=1e-6, atol=0) and iters <= 16   # exact after one step; checked per batch of 16


def test_densify_undetermined_regions_stay_zero(env):
    ds = np.zeros((6, 10), np.float32); ds[2, 1] = 1.0
    s = np.zeros((6, 10), np.float32); s[:, 5:] = 1.0
    x, _ = _solve(env, ds, None, s, np.ones((6, 10), np.float32), None, tol=1e-7)
    assert np.allclose(x[:, :6], 1.0, rtol=1e-5) and (x[:, 6:] == 0).all()


def test_densify_one_launch_and_per_iteration_launches_agree(env):
    # a frame that spreads over every multiprocessor (several blocks, halo
    # bands crossing rows): both solvers reach the tolerance, stop within one
    # batch of iterations of each other and agree with the direct solve
    rng = np.random.default_rng(11)
    H, W = 270, 480
    ds, B, mf, mi, dp = _inputs(rng, H, W, 0.3)
    x0, (i0, r0) = _solve(env, ds, B, mf, mi, dp, tol=1e-6, max_iters=20000, solver=0)
    x1, (i1, r1) = _solve(env, ds, B, mf, mi, dp, tol=1e-6, max_iters=20000, solver=1)
    p = DN.DenseParams()
    want = DN.densify(ds.astype(np.float64), B, mf, mi, dp.astype(np.float64), p)
    for name, x, rel in (("one launch", x0, r0), ("per-iteration launches", x1, r1)):
        assert rel <= 1e-6, name
        assert _true_relres(x, ds, B, mf, mi, dp, p) <= 2.5e-6, name
        err = np.abs(x - want).max() / np.abs(want).max()
        assert err <= 1e-3, (name, err)
        assert (x[want == 0] == 0).all(), name
    assert abs(i0 - i1) <= 16, (i0, i1)


def test_densify_a_stereo_depth_map(env):
    # the sparse depth of the quarter-size path, a contour where the ground
    # truth jumps, texture weights from the image gradient
    torch, binding, st = env
    s = scenes.plane_scene(320, 240, 64, 6, seed=scenes.seed_for(2, 960), drange=(4, 56), slanted=True,
                           noise_sigma=2.0)
    z = st.depth(_dev(torch, s.left), _dev(torch, s.right), 32, 700.0, 0.12).cpu().numpy()
    g = s.disp
    B = ((np.abs(np.diff(g, axis=1, append=g[:, -1:])) > 1) | (np.abs(np.diff(g, axis=0, append=g[-1:])) > 1))
    Y = s.left.astype(np.float32).mean(axis=2)
    gm = np.hypot(*np.gradient(Y))
    mi = (gm / gm.max()).astype(np.float32)
    mf = np.ones_like(mi)
    x, (iters, rel) = _solve(env, z, B.astype(np.uint8), mf, mi, None, tol=1e-6, max_iters=20000)
    want = DN.densify(z.astype(np.float64), B.astype(np.uint8), mf, mi, None)
    assert rel <= 1e-6
    assert _true_relres(x, z, B.astype(np.uint8), mf, mi, None, DN.DenseParams()) <= 1e-5
    assert np.abs(x - want).max() <= 1e-3 * np.abs(want).max()
    assert (x > 0).mean() > (z > 0).mean()


def test_densify_rejects_bad_arguments(env):
    torch, binding, st = env
    d = torch.zeros((4, 4), dtype=torch.float32, device="cuda")
    for over in (dict(tol=0.0), dict(lambda_s=-1.0), dict(max_iters=-1), dict(solver=2), dict(solver=-1)):
        with pytest.raises(binding.DcoError) as e:
            st.densify(d, params=binding.DenseParams.default(**over))
        assert e.value.code == binding.DCO_EINVAL
