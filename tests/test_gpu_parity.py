"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Every input is a seeded synthetic scene (paper_2203_02300_gb300.scenes).
Tolerances: tests/parity.py.
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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def oparams(bp):
    """oracle Params equal to a binding Params."""
    return O.Params(lambda_ad=float(bp.lambda_ad), lambda_census=float(bp.lambda_census),
                    gamma_l=float(bp.gamma_l), eps=float(bp.eps), census_w=bp.census_w,
                    census_h=bp.census_h, arm_l1=bp.arm_l1, arm_l2=bp.arm_l2, tau1=bp.tau1,
                    tau2=bp.tau2, lr_tol=bp.lr_tol, smooth_arms=bp.smooth_arms,
                    agg_order=bp.agg_order, d_min=bp.d_min)


def run_views(env, left, right, D, bp=None):
    torch, binding, st = env
    out, dl, dr, cl, cr = st.match_views(dev(torch, left), dev(torch, right), D, bp)
    torch.cuda.synchronize()
    st.sync_status()
    return (out.cpu().numpy(), dl.cpu().numpy(), dr.cpu().numpy(), cl.cpu().numpy(), cr.cpu().numpy())


def full_check(env, left, right, D, bp=None, rows=None, label=None):
    """The GPU's two disparity maps, minimum costs and checked map against
    the FP64 oracle under the parity rule (near ties excused, <= 0.1 %)."""
    torch, binding, st = env
    op = oparams(bp) if bp is not None else O.Params()
    out, dl, dr, cl, cr = run_views(env, left, right, D, bp)
    ref = O.match(left, right, D, op, rows=rows, quantized=True)
    sl = slice(*rows) if rows else slice(None)
    H, W, _ = left.shape
    label = label or f"{W}x{H} D={D}"
    if rows:
        label += f" rows {rows[0]}-{rows[1]}"
    n = parity.check_disparity(dl[sl], ref.disp_l, ref.best_l, ref.second_l, f"{label} left disparity", ref.qdisp_l)
    n += parity.check_disparity(dr[sl], ref.disp_r, ref.best_r, ref.second_r, f"{label} right disparity",
                                ref.qdisp_r)
    parity.check_cost(cl[sl], ref.best_l, dl[sl], ref.disp_l, f"{label} left cost")
    parity.check_cost(cr[sl], ref.best_r, dr[sl], ref.disp_r, f"{label} right cost")
    assert (out == O.lr_check(dl, dr, op.lr_tol)).all(), "consistency map"
    parity.check_final(out[sl], ref, f"{label} final map")
    return n, out, dl, dr


# --------------------------------------------------------------- stages
def stage_images():
    s1 = scenes.config_scene(1)
    s2 = scenes.config_scene(2)
    rnd = [scenes.random_pair(w, h, 100 + w)[0] for (w, h) in ((1, 1), (7, 5), (33, 17), (130, 3))]
    flat = np.full((20, 50, 3), 128, np.uint8)
    return [s1.left, s1.right, s2.left] + rnd + [flat]


@pytest.mark.parametrize("k", range(8))
def test_census_bit_exact(env, k):
    torch, binding, st = env
    img = stage_images()[k]
    got = st.census(dev(torch, img)).cpu().numpy().view(np.uint64)
    assert (got == O.census(img)).all()


@pytest.mark.parametrize("k", range(8))
def test_arms_bit_exact(env, k):
    torch, binding, st = env
    img = stage_images()[k]
    got = st.arms(dev(torch, img)).cpu().numpy()
    assert (got == O.arms(img)).all()


@pytest.mark.parametrize("k", range(8))
def test_smoothed_arms_bit_exact(env, k):
    # Sect. 4.1 smoothing (3x3 opening): integer work, bit-exact
    torch, binding, st = env
    img = stage_images()[k]
    bp = binding.Params.default(smooth_arms=1)
    got = st.arms(dev(torch, img), bp).cpu().numpy()
    assert np.array_equal(got, O.arms(img, oparams(bp)))


def test_census_and_arms_other_windows(env):
    torch, binding, st = env
    img = scenes.config_scene(1).left
    for cw, ch, l1, l2, t1, t2 in ((7, 5, 10, 4, 15, 5), (11, 5, 40, 20, 30, 8), (1, 1, 1, 0, 256, 256),
                                   (9, 7, 34, 17, 0, 6), (9, 7, 34, 2, 255, 0), (3, 3, 8, 8, 1, 1)):
        bp = binding.Params.default(census_w=cw, census_h=ch, arm_l1=l1, arm_l2=l2, tau1=t1, tau2=t2)
        got = st.census(dev(torch, img), bp).cpu().numpy().view(np.uint64)
        assert (got == O.census(img, cw, ch)).all()
        got = st.arms(dev(torch, img), bp).cpu().numpy()
        assert (got == O.arms(img, oparams(bp))).all()


def test_lr_check_stage(env):
    torch, binding, st = env
    rng = np.random.default_rng(21)
    dl = rng.integers(0, 9, (31, 45)).astype(np.int16)
    dr = rng.integers(0, 9, (31, 45)).astype(np.int16)
    for tol in (-1, 0, 1, 3):
        got = st.lr_check(dev(torch, dl), dev(torch, dr), tol).cpu().numpy()
        assert (got == O.lr_check(dl, dr, tol)).all()


# ----------------------------------------------------------- full path
def test_config1_full_parity(env):
    s = scenes.config_scene(1)
    n, out, dl, dr = full_check(env, s.left, s.right, s.D, label="config 1 (320x240 D=32)")
    gt = np.rint(s.disp).astype(np.int16)
    assert ((dl == gt) & ~s.occluded).sum() / (~s.occluded).sum() > 0.99


def test_config2_full_parity(env):
    s = scenes.config_scene(2)
    full_check(env, s.left, s.right, s.D, label="config 2 (640x480 D=64)")


@pytest.mark.parametrize("config", [1, 2])
def test_lr_check_rejects_ground_truth_occlusions(env, config):
    # outlier removal (Sect. 4.3): of the left pixels the scene generator
    # marks occluded (no visible match in the right view), the fraction the
    # consistency check rejects; and the fraction of visible pixels it keeps
    s = scenes.config_scene(config)
    out, dl, dr, cl, cr = run_views(env, s.left, s.right, s.D)
    occ = s.occluded
    rejected = float((out[occ] < 0).mean())
    kept = float((out[~occ] >= 0).mean())
    parity.note(f"config {config}: the consistency check rejects {100 * rejected:.1f} % of the "
                f"{int(occ.sum())} ground-truth occluded pixels and keeps {100 * kept:.1f} % of the visible ones")
    assert rejected > 0.3 and kept > 0.7


def test_config1_cost_volume_both_views(env):
    torch, binding, st = env
    s = scenes.config_scene(1)
    ref = O.match(s.left, s.right, s.D, volume=True)
    L, R = dev(torch, s.left), dev(torch, s.right)
    for view, want in ((0, ref.vol_l), (1, ref.vol_r)):
        got = st.cost_volume(L, R, s.D, view).cpu().numpy()
        parity.check_volume(got, want, f"volume view {view}")


@pytest.mark.parametrize("W,H,D", [(1, 1, 1), (7, 5, 3), (33, 17, 16), (100, 3, 40), (65, 40, 33),
                                   (300, 40, 256), (64, 64, 64), (97, 71, 50)])
def test_ragged_sizes(env, W, H, D):
    s = scenes.plane_scene(W, H, D, 3, seed=1000 + W * H + D, drange=(0, max(0, min(D - 1, W - 1))),
                           noise_sigma=1.0) if W >= 8 and H >= 8 else None
    if s is None:
        left, right = scenes.random_pair(W, H, 7 * W + H)
    else:
        left, right = s.left, s.right
    full_check(env, left, right, D)


def test_maximum_width(env):
    # the widest rows (16384 columns: 32 first-pass blocks of 512 per row) at
    # the largest range D = 256
    s = scenes.plane_scene(16384, 12, 256, 40, seed=scenes.seed_for(1, 500), drange=(2, 250), noise_sigma=2.0)
    full_check(env, s.left, s.right, 256, label="16384x12 D=256")


def test_maximum_height(env):
    # the tallest columns (16384 rows: 38 second-pass blocks per column),
    # sampled row bands against the oracle (census and arms of the whole image)
    torch, binding, st = env
    s = scenes.plane_scene(48, 16384, 24, 30, seed=scenes.seed_for(1, 501), drange=(2, 22), noise_sigma=2.0)
    out, dl, dr, cl, cr = run_views(env, s.left, s.right, 24)
    tl, tr, tf = (parity.Tally(f"48x16384 D=24 {v}") for v in ("left disparity", "right disparity", "final map"))
    for rows in ((0, 48), (8170, 8218), (16336, 16384)):
        ref = O.match(s.left, s.right, 24, rows=rows, quantized=True)
        sl = slice(*rows)
        what = f"48x16384 rows {rows[0]}-{rows[1]}"
        parity.check_disparity(dl[sl], ref.disp_l, ref.best_l, ref.second_l, what + " left", ref.qdisp_l, tally=tl)
        parity.check_disparity(dr[sl], ref.disp_r, ref.best_r, ref.second_r, what + " right", ref.qdisp_r, tally=tr)
        parity.check_cost(cl[sl], ref.best_l, dl[sl], ref.disp_l)
        parity.check_cost(cr[sl], ref.best_r, dr[sl], ref.disp_r)
        parity.check_final(out[sl], ref, what + " final map", tally=tf)
    for t in (tl, tr, tf):
        t.close()


@pytest.mark.parametrize("chunk", [1, 5, 16, 32, 33, 64])
def test_passes_are_bit_identical(env, chunk):
    torch, binding, st = env
    s = scenes.config_scene(1)
    base = run_views(env, s.left, s.right, s.D)
    got = run_views(env, s.left, s.right, s.D, binding.Params.default(d_chunk=chunk))
    for a, b in zip(base, got):
        assert np.array_equal(a, b)


def test_identical_views(env):
    rng = np.random.default_rng(31)
    img = np.clip(np.rint(scenes._texture(rng, 60, 90)), 0, 255).astype(np.uint8)
    out, dl, dr, cl, cr = run_views(env, img, img, 24)
    assert (dl == 0).all() and (dr == 0).all() and (out == 0).all()
    assert (cl == 0).all() and (cr == 0).all()


@pytest.mark.parametrize("over", [dict(lr_tol=-1), dict(lr_tol=0), dict(arm_l1=5, arm_l2=2),
                                  dict(gamma_l=3.0, eps=0.5), dict(lambda_ad=30.0, lambda_census=15.0),
                                  dict(census_w=7, census_h=5), dict(arm_l1=40, arm_l2=40, tau1=256, tau2=256),
                                  dict(smooth_arms=1), dict(smooth_arms=1, arm_l1=5, arm_l2=2)])
def test_parameter_variants(env, over):
    torch, binding, st = env
    s = scenes.config_scene(1)
    full_check(env, s.left, s.right, s.D, binding.Params.default(**over))


# ------------------------------------------- the other aggregation order
# region = union over q on p's horizontal arm of q's vertical segment
# (k_vcost column sums, then k_vagg scanning rows)
def test_vh_order_config1_full_parity(env):
    torch, binding, st = env
    s = scenes.config_scene(1)
    n, out, dl, dr = full_check(env, s.left, s.right, s.D, binding.Params.default(agg_order=1))
    gt = np.rint(s.disp).astype(np.int16)
    assert ((dl == gt) & ~s.occluded).sum() / (~s.occluded).sum() > 0.99


@pytest.mark.parametrize("over", [dict(agg_order=1), dict(smooth_arms=1), dict(agg_order=1, smooth_arms=1)])
def test_config2_variants_full_parity(env, over):
    # the V-then-H order and the smoothed window on the whole 640x480 D=64
    # frame of the metric's workload
    torch, binding, st = env
    s = scenes.config_scene(2)
    full_check(env, s.left, s.right, s.D, binding.Params.default(**over), label=f"config 2 {over}")


def test_vh_order_differs_from_hv_order(env):
    # the two regions differ wherever arms of neighbours differ: the costs
    # must not be equal everywhere (guards against a silent order-0 run)
    torch, binding, st = env
    s = scenes.config_scene(1)
    a = run_views(env, s.left, s.right, s.D)
    b = run_views(env, s.left, s.right, s.D, binding.Params.default(agg_order=1))
    assert not np.array_equal(a[3], b[3])


# (D <= W is a library rule); 20x1100: columns longer than one k_vcost chunk
@pytest.mark.parametrize("W,H,D", [(1, 1, 1), (7, 5, 3), (33, 17, 16), (3, 100, 3), (100, 3, 40),
                                   (40, 65, 33), (97, 71, 50), (600, 20, 64), (20, 1100, 16)])
def test_vh_order_ragged_sizes(env, W, H, D):
    torch, binding, st = env
    s = scenes.plane_scene(W, H, D, 3, seed=2000 + W * H + D, drange=(0, max(0, min(D - 1, W - 1))),
                           noise_sigma=1.0) if W >= 8 and H >= 8 else None
    if s is None:
        left, right = scenes.random_pair(W, H, 11 * W + H)
    else:
        left, right = s.left, s.right
    full_check(env, left, right, D, binding.Params.default(agg_order=1))


@pytest.mark.parametrize("over", [dict(d_chunk=5), dict(d_chunk=33), dict(smooth_arms=1),
                                  dict(arm_l1=5, arm_l2=2), dict(arm_l1=40, arm_l2=40, tau1=256, tau2=256)])
def test_vh_order_variants(env, over):
    torch, binding, st = env
    s = scenes.config_scene(1)
    full_check(env, s.left, s.right, s.D, binding.Params.default(agg_order=1, **over))


def test_vh_order_cost_volume(env):
    torch, binding, st = env
    s = scenes.config_scene(1)
    ref = O.match(s.left, s.right, s.D, O.Params(agg_order=1), volume=True)
    L, R = dev(torch, s.left), dev(torch, s.right)
    got = st.cost_volume(L, R, s.D, 0, binding.Params.default(agg_order=1)).cpu().numpy()
    parity.check_volume(got, ref.vol_l, "volume view 0, order 1")


def test_config5_full_frame(env):
    # one 1920x1080 D=256 pair (32 planes, 200 discs, sigma 3) whole, against
    # the FP64 oracle (about a billion FP64 evaluations on the host cores)
    torch, binding, st = env
    s = scenes.config_scene(5)
    out, dl, dr, cl, cr = run_views(env, s.left, s.right, s.D)
    ref = O.match(s.left, s.right, s.D)
    what = "config 5 pair 0 (1920x1080 D=256) full frame"
    parity.check_disparity(dl, ref.disp_l, ref.best_l, ref.second_l, what + " left disparity")
    parity.check_disparity(dr, ref.disp_r, ref.best_r, ref.second_r, what + " right disparity")
    parity.check_cost(cl, ref.best_l, dl, ref.disp_l, what + " left cost")
    parity.check_cost(cr, ref.best_r, dr, ref.disp_r, what + " right cost")
    parity.check_final(out, ref, what + " final map")


def test_vh_order_config5_sampled_rows(env):
    # 1920x1080 D=256: k_vcost sums the 1080-row columns in chunks of 512
    # rows (rows 509..515 straddle the first boundary), k_vagg scans the
    # 1920-column rows in several chunks
    torch, binding, st = env
    s = scenes.config_scene(5)
    bp = binding.Params.default(agg_order=1)
    out, dl, dr, cl, cr = run_views(env, s.left, s.right, s.D, bp)
    tl, tr, tf = (parity.Tally(f"config 5 V-then-H order {v}") for v in ("left disparity", "right disparity",
                                                                          "final map"))
    for rows in ((0, 6), (509, 515), (1074, 1080)):
        ref = O.match(s.left, s.right, s.D, O.Params(agg_order=1), rows=rows, quantized=True)
        sl = slice(*rows)
        what = f"config 5 V-then-H order rows {rows[0]}-{rows[1]}"
        parity.check_disparity(dl[sl], ref.disp_l, ref.best_l, ref.second_l, what + " left disparity", ref.qdisp_l,
                               tally=tl)
        parity.check_disparity(dr[sl], ref.disp_r, ref.best_r, ref.second_r, what + " right disparity",
                               ref.qdisp_r, tally=tr)
        parity.check_cost(cl[sl], ref.best_l, dl[sl], ref.disp_l)
        parity.check_cost(cr[sl], ref.best_r, dr[sl], ref.disp_r)
        parity.check_final(out[sl], ref, what + " final map", tally=tf)
    for t in (tl, tr, tf):
        t.close()


# --------------------------------------------------------------- tile shapes
@pytest.mark.parametrize("order", [0, 1])
def test_tile_shapes_change_nothing(env, order):
    # blocks of the two 1-D passes (h_chunk, v_chunk) from 32 positions to
    # whole lines, with and without narrow passes: every map and cost equals
    # the automatic tiles' bit for bit, and the oracle's parity rule holds
    torch, binding, st = env
    s = scenes.config_scene(2)
    auto = run_views(env, s.left, s.right, s.D, binding.Params.default(agg_order=order))
    for d, h, v in ((0, 32, 0), (0, 0, 32), (0, 96, 100), (32, 320, 240), (0, 224, 160), (48, 600, 479),
                    (0, 16384, 16384), (0, 1000, 0)):
        got = run_views(env, s.left, s.right, s.D,
                        binding.Params.default(agg_order=order, d_chunk=d, h_chunk=h, v_chunk=v))
        for a, b in zip(got, auto):
            assert np.array_equal(a, b), (d, h, v)
    full_check(env, s.left, s.right, s.D, binding.Params.default(agg_order=order, h_chunk=96, v_chunk=100),
               label=f"config 2 order {order} tiles 96 x 100")


def test_tile_shapes_config5_rows(env):
    # 1920 x 1080: first-pass blocks of 288 and 640 columns, second-pass
    # blocks of 135 and 270 rows against the automatic (512, 360)
    torch, binding, st = env
    s = scenes.config_scene(5)
    L, R = dev(torch, s.left), dev(torch, s.right)
    auto = st.match(L, R, s.D).cpu().numpy()
    for h, v in ((288, 135), (640, 270)):
        got = st.match(L, R, s.D, binding.Params.default(h_chunk=h, v_chunk=v)).cpu().numpy()
        assert np.array_equal(got, auto), (h, v)


# --------------------------------------------------------------- Eq. 3 range [d_min, d_max]
@pytest.mark.parametrize("W,H,dmin,D,over", [(160, 96, 16, 48, {}), (200, 80, 5, 37, dict(d_chunk=32)),
                                             (160, 96, 3, 29, dict(agg_order=1)), (320, 64, 200, 56, {}),
                                             (96, 40, 40, 2, {}), (130, 70, 9, 70, dict(d_chunk=33))])
def test_d_min_search(env, W, H, dmin, D, over):
    # passes start at d_min (a ragged last pass where D is not a multiple of
    # the pass width), maps hold absolute disparities, the largest range
    # reaches d = 255 (the padded candidate rows)
    torch, binding, st = env
    s = scenes.plane_scene(W, H, dmin + D, 4, seed=scenes.seed_for(1, 400 + dmin + D),
                           drange=(dmin + min(2, D - 1), dmin + max(min(2, D - 1), D - 3)), noise_sigma=2.0)
    bp = binding.Params.default(d_min=dmin, **over)
    n, out, dl, dr = full_check(env, s.left, s.right, D, bp, label=f"{W}x{H} d in [{dmin}, {dmin + D - 1}]")
    for m in (dl, dr):
        assert ((m >= dmin) & (m < dmin + D)).all()


def test_d_min_cost_volume(env):
    torch, binding, st = env
    s = scenes.plane_scene(128, 64, 40, 3, seed=scenes.seed_for(1, 410), drange=(12, 36))
    for view in (0, 1):
        for order in (0, 1):
            ref = O.match(s.left, s.right, 30, O.Params(d_min=10, agg_order=order), volume=True)
            got = st.cost_volume(dev(torch, s.left), dev(torch, s.right), 30, view,
                                 binding.Params.default(d_min=10, agg_order=order)).cpu().numpy()
            parity.check_volume(got, ref.vol_r if view else ref.vol_l, f"volume view {view} order {order}, d_min 10")


def test_d_min_vote(env):
    # Eq. 4 over [d_min, d_max]: values below d_min neither vote nor survive
    torch, binding, st = env
    rng = np.random.default_rng(41)
    s = scenes.plane_scene(150, 90, 60, 5, seed=scenes.seed_for(1, 420), drange=(22, 58))
    d = np.clip(np.rint(s.disp), 0, 59).astype(np.int16)
    u = rng.random(d.shape)
    d[u < 0.15] = rng.integers(0, 60, int((u < 0.15).sum()))
    d[(u >= 0.15) & (u < 0.25)] = -1
    for dmin, D, it in ((20, 40, 2), (7, 33, 1)):
        got = st.vote(dev(torch, s.left), dev(torch, d), D,
                      binding.Params.default(d_min=dmin, vote_iters=it)).cpu().numpy()
        st.sync_status()
        assert np.array_equal(got, O.vote(d, O.arms(s.left), D, it, d_min=dmin))


def test_d_min_batch_equals_single(env):
    torch, binding, st = env
    bp = binding.Params.default(d_min=12)
    sc = [scenes.plane_scene(w, h, 12 + D, 3, seed=scenes.seed_for(1, 430 + w), drange=(14, 10 + D))
          for (w, h, D) in ((160, 96, 40), (97, 61, 20), (256, 40, 64))]
    pairs = [(dev(torch, x.left), dev(torch, x.right), x.D - 12, torch.empty((x.left.shape[0], x.left.shape[1]),
                                                                              dtype=torch.int16, device="cuda"))
             for x in sc]
    st.match_batch(pairs, bp)
    torch.cuda.synchronize()
    for (l, r, D, o) in pairs:
        assert np.array_equal(o.cpu().numpy(), st.match(l, r, D, bp).cpu().numpy())


def _scenes_in_pool(config, items):
    # scene generation is plain NumPy on the host; a spawned pool (safe after
    # CUDA initialisation) renders the 1920x1080 scenes in parallel
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(min(len(items), 8), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(scenes.config_scene, [config] * len(items), items))


CONFIG5_BUDGET = 1_500_000_000   # bytes: below one 2.12 GB FP32 volume of one view


def test_config5_batch_of_8_under_a_budget(env):
    # 8 pairs of 1920x1080, D = 256 on a handle whose workspace budget is
    # below one materialised volume: the batch is admitted in groups that fit
    # (passes of 32 disparities), the allocation never exceeds the budget,
    # every map equals the pair matched alone, and two pairs are checked
    # against the FP64 oracle on row bands (borders and middle)
    torch, binding, st = env
    ss = _scenes_in_pool(5, list(range(8)))
    assert CONFIG5_BUDGET < 1920 * 1080 * 256 * 4
    pairs = [(dev(torch, s.left), dev(torch, s.right), s.D,
              torch.full((s.H, s.W), -9, dtype=torch.int16, device="cuda")) for s in ss]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with binding.Stereo(0, budget_bytes=CONFIG5_BUDGET) as h:
        h.match_batch(pairs)
        h.stream_status()
        free1 = torch.cuda.mem_get_info()[0]
        assert 0 < h.workspace_allocated() <= CONFIG5_BUDGET
        assert free0 - free1 <= CONFIG5_BUDGET
        assert h.batch_groups() > 1
    bands = ((0, 6), (537, 543), (1074, 1080))
    tl, tr, tf = (parity.Tally(f"config 5 (1920x1080 D=256) {v}") for v in ("left disparity", "right disparity",
                                                                             "final map"))
    for k, (s, (L, R, D, out)) in enumerate(zip(ss, pairs)):
        got = out.cpu().numpy()
        if k >= 2:
            assert np.array_equal(got, st.match(L, R, D).cpu().numpy()), k
            continue
        fo, dl, dr, cl, cr = run_views(env, s.left, s.right, s.D)
        assert np.array_equal(got, fo), k
        assert (fo == O.lr_check(dl, dr, 1)).all()
        for rows in bands[k:k + 2]:
            ref = O.match(s.left, s.right, s.D, rows=rows, quantized=True)
            sl = slice(*rows)
            what = f"config 5 (1920x1080 D=256) pair {k} rows {rows[0]}-{rows[1]}"
            parity.check_disparity(dl[sl], ref.disp_l, ref.best_l, ref.second_l, what + " left disparity",
                                   ref.qdisp_l, tally=tl)
            parity.check_disparity(dr[sl], ref.disp_r, ref.best_r, ref.second_r, what + " right disparity",
                                   ref.qdisp_r, tally=tr)
            parity.check_cost(cl[sl], ref.best_l, dl[sl], ref.disp_l, what + " left cost")
            parity.check_cost(cr[sl], ref.best_r, dr[sl], ref.disp_r, what + " right cost")
            parity.check_final(got[sl], ref, what + " final map", tally=tf)
    for t in (tl, tr, tf):
        t.close()


def test_batch_single_pair_beyond_the_budget_is_rejected(env):
    torch, binding, st = env
    s = scenes.config_scene(1)
    need = binding.Stereo.workspace_bytes(s.W, s.H, s.D, binding.Params.default(d_chunk=32))
    with binding.Stereo(0, budget_bytes=need - 1) as h:
        out = torch.full((s.H, s.W), -9, dtype=torch.int16, device="cuda")
        with pytest.raises(binding.DcoError) as e:
            h.match_batch([(dev(torch, s.left), dev(torch, s.right), s.D, out)] * 2)
        assert e.value.code == binding.DCO_EBUDGET
        assert h.workspace_allocated() == 0
        torch.cuda.synchronize()
        assert (out == -9).all()


def test_match_host_equals_device_path(env):
    # pageable buffers (staging copies), pinned buffers (read and written in
    # place by the kernels) and pinned buffers with Eq. 4 rounds (staged map)
    torch, binding, st = env
    s = scenes.config_scene(2)
    out = st.match(dev(torch, s.left), dev(torch, s.right), s.D).cpu().numpy()
    assert np.array_equal(out, st.match_host(s.left, s.right, s.D))
    Lp = torch.from_numpy(s.left).pin_memory().numpy()
    Rp = torch.from_numpy(s.right).pin_memory().numpy()
    op = torch.full((s.H, s.W), -7, dtype=torch.int16).pin_memory().numpy()
    assert np.array_equal(out, st.match_host(Lp, Rp, s.D, out=op))
    pv = binding.Params.default(vote_iters=1)
    want = st.match(dev(torch, s.left), dev(torch, s.right), s.D, pv).cpu().numpy()
    assert np.array_equal(want, st.match_host(Lp, Rp, s.D, pv, out=op))


@pytest.mark.parametrize("config", [1, 2])
def test_mirror_swap_symmetry_on_the_gpu(env, config):
    # swapping the views and mirroring both rows exchanges the two reference
    # views: the kernels' integer region sums run the other way along the
    # rows and give the same fixed-point values, so the maps mirror exactly
    torch, binding, st = env
    s = scenes.config_scene(config)
    out, dl, dr, cl, cr = run_views(env, s.left, s.right, s.D)
    mout, mdl, mdr, mcl, mcr = run_views(env, s.right[:, ::-1], s.left[:, ::-1], s.D)
    assert np.array_equal(mdl, dr[:, ::-1]) and np.array_equal(mdr, dl[:, ::-1])
    assert np.array_equal(mcl, cr[:, ::-1]) and np.array_equal(mcr, cl[:, ::-1])


def test_repeat_runs_bit_identical(env):
    s = scenes.config_scene(2)
    a = run_views(env, s.left, s.right, s.D)
    b = run_views(env, s.left, s.right, s.D)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ----------------------------------------------------------- errors
def test_argument_errors(env):
    torch, binding, st = env
    L = dev(torch, np.zeros((8, 8, 3), np.uint8))
    out = torch.empty((8, 8), dtype=torch.int16, device="cuda")
    lib = binding.lib()
    h = st._h
    s0 = torch.cuda.current_stream().cuda_stream
    assert lib.dco_stereo_match(h, L.data_ptr(), L.data_ptr(), 8, 8, 9, None, out.data_ptr(), s0) == binding.DCO_EINVAL
    assert lib.dco_stereo_match(h, L.data_ptr(), L.data_ptr(), 8, 8, 0, None, out.data_ptr(), s0) == binding.DCO_EINVAL
    assert lib.dco_stereo_match(h, L.data_ptr(), L.data_ptr(), 0, 8, 1, None, out.data_ptr(), s0) == binding.DCO_EINVAL
    assert lib.dco_stereo_match(h, None, L.data_ptr(), 8, 8, 4, None, out.data_ptr(), s0) == binding.DCO_EINVAL
    assert lib.dco_stereo_match(h, L.data_ptr(), L.data_ptr(), 8, 8, 4, None, None, s0) == binding.DCO_EINVAL
    assert lib.dco_stereo_match(None, L.data_ptr(), L.data_ptr(), 8, 8, 4, None, out.data_ptr(), s0) == binding.DCO_EINVAL
    assert lib.dco_stereo_match(h, L.data_ptr(), L.data_ptr(), 8, 0, 1, None, out.data_ptr(), s0) == binding.DCO_EINVAL
    assert lib.dco_stereo_match(h, L.data_ptr(), L.data_ptr(), 16385, 1, 1, None, out.data_ptr(),
                                s0) == binding.DCO_EINVAL
    for bad in (dict(census_w=8), dict(census_w=13, census_h=7), dict(arm_l1=41), dict(arm_l1=0),
                dict(lambda_ad=0.0), dict(eps=-1.0), dict(d_chunk=-1), dict(d_min=-1), dict(d_min=5),
                dict(h_chunk=8), dict(v_chunk=-2)):
        p = binding.Params.default(**bad)
        import ctypes
        assert lib.dco_stereo_match(h, L.data_ptr(), L.data_ptr(), 8, 8, 4, ctypes.byref(p), out.data_ptr(),
                                    s0) == binding.DCO_EINVAL, bad
    st.sync_status()


def test_budget_rejects_before_launch(env):
    torch, binding, st = env
    s = scenes.config_scene(1)
    small = binding.Stereo(0, budget_bytes=1 << 20)
    with pytest.raises(binding.DcoError) as e:
        small.match(dev(torch, s.left), dev(torch, s.right), s.D)
    assert e.value.code == binding.DCO_EBUDGET
    # a budget that fits per-pixel buffers plus one 32-disparity pass works
    need = binding.Stereo.workspace_bytes(s.W, s.H, s.D, binding.Params.default(d_chunk=32))
    mid = binding.Stereo(0, budget_bytes=need)
    out = mid.match(dev(torch, s.left), dev(torch, s.right), s.D).cpu().numpy()
    ref = st.match(dev(torch, s.left), dev(torch, s.right), s.D).cpu().numpy()
    assert np.array_equal(out, ref)
    small.close()
    mid.close()
