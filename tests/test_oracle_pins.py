"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formula: each checks a closed form at a
point, an invariant, a special case that reduces to a textbook or library
routine, or a brute-force re-derivation on tiny inputs, chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
swapped view, a transposed bit order) fails at least one of them.
"""
import itertools

import numpy as np
import pytest
import sympy

from oracle import oracle as O
from paper_2203_02300_gb300 import scenes

P = O.Params()


def grey_image(v):
    v = np.asarray(v, np.uint8)
    return np.repeat(v[:, :, None], 3, axis=2)


# ----------------------------------------------------------------- grey
def test_grey_closed_forms():
    img = np.array([[[255, 255, 255], [0, 0, 0], [255, 0, 0], [0, 255, 0], [0, 0, 255]]], np.uint8)
    # (77*255+128)>>8 = 77, (150*255+128)>>8 = 149, (29*255+128)>>8 = 29
    assert O.grey(img).tolist() == [[255, 0, 77, 149, 29]]


def test_grey_matches_bt601_luma_within_one():
    rng = np.random.default_rng(1)
    img = rng.integers(0, 256, (37, 53, 3), dtype=np.uint8)
    f = img.astype(np.float64)
    luma = 0.299 * f[..., 0] + 0.587 * f[..., 1] + 0.114 * f[..., 2]
    assert np.abs(O.grey(img) - luma).max() <= 1.0


def test_grey_of_neutral_pixels_is_identity():
    v = np.arange(256, dtype=np.uint8).reshape(16, 16)
    assert (O.grey(grey_image(v)) == v).all()


# --------------------------------------------------------------- census
def test_census_constant_image_is_zero():
    for c in (0, 17, 255):
        img = np.full((11, 13, 3), c, np.uint8)
        assert (O.census(img) == 0).all()


def _kindex(dy, dx, cw=9, ch=7):
    """Bit position of window offset (dy, dx): rows top to bottom, columns left
    to right, centre skipped."""
    k = (dy + ch // 2) * cw + (dx + cw // 2)
    return k - 1 if (dy, dx) > (0, 0) else k


def test_census_ramp_sets_exactly_the_earlier_half():
    # Y = 12*y + x: a neighbour is darker iff it comes before p in row-major
    # order, so the interior census is the 31 low bits.
    H, W = 14, 20
    v = 12 * np.arange(H)[:, None] + np.arange(W)[None, :]
    c = O.census(grey_image(v))
    interior = c[3:H - 3, 4:W - 4]
    assert (interior == np.uint64((1 << 31) - 1)).all()
    # top-left: every clamped neighbour is >= p -> no bit; bottom-right:
    # the 19 offsets with dy >= 0 and dx >= 0 clamp onto p itself.
    assert int(c[0, 0]) == 0
    assert bin(int(c[H - 1, W - 1])).count("1") == 62 - 19


def test_census_dark_impulse_gives_one_bit_at_its_offset():
    H, W = 15, 17
    v = np.full((H, W), 200, np.uint8)
    y0, x0 = 7, 8
    v[y0, x0] = 10
    c = O.census(grey_image(v))
    for y in range(H):
        for x in range(W):
            dy, dx = y0 - y, x0 - x
            if (y, x) == (y0, x0):
                assert int(c[y, x]) == 0
            elif abs(dy) <= 3 and abs(dx) <= 4:
                assert int(c[y, x]) == 1 << _kindex(dy, dx), (y, x)
            else:
                assert int(c[y, x]) == 0


def test_census_bright_impulse_sets_all_62_bits():
    v = np.zeros((9, 11), np.uint8)
    v[4, 5] = 200
    c = O.census(grey_image(v))
    assert int(c[4, 5]) == (1 << 62) - 1
    c2 = c.copy()
    c2[4, 5] = 0
    assert (c2 == 0).all()


def test_census_invariant_under_monotone_grey_map():
    rng = np.random.default_rng(3)
    v = rng.integers(0, 128, (23, 29), dtype=np.uint8)
    assert (O.census(grey_image(v)) == O.census(grey_image(2 * v + 1))).all()


def test_hamming_counts_bits():
    rng = np.random.default_rng(4)
    for a, b in rng.integers(0, 2 ** 63, (200, 2), dtype=np.int64):
        a, b = int(a) * 2 + 1, int(b)
        assert O.hamming(a, b) == bin(a ^ b).count("1")


# ----------------------------------------------------------------- arms
def brute_arm(img, x, y, ex, ey, p):
    """Largest k for which ALL of the double-threshold conditions hold for
    every j <= k, checked from scratch for each candidate k."""
    H, W, _ = img.shape
    f = img.astype(int)
    best = 0
    for k in range(1, p.arm_l1 + 1):
        ok = True
        for j in range(1, k + 1):
            qx, qy = x + j * ex, y + j * ey
            if not (0 <= qx < W and 0 <= qy < H):
                ok = False
                break
            dp = np.abs(f[qy, qx] - f[y, x]).max()
            dn = np.abs(f[qy, qx] - f[qy - ey, qx - ex]).max()
            if dp >= p.tau1 or dn >= p.tau1 or (j > p.arm_l2 and dp >= p.tau2):
                ok = False
                break
        if ok:
            best = k
    return best


def test_arms_match_brute_force_on_blocky_images():
    rng = np.random.default_rng(5)
    p = O.Params(arm_l1=7, arm_l2=3, tau1=20, tau2=6)
    for trial in range(3):
        base = rng.integers(0, 256, (4, 5, 3))
        img = np.kron(base, np.ones((4, 4, 1))).astype(np.int64)
        img = np.clip(img + rng.integers(-6, 7, img.shape), 0, 255).astype(np.uint8)
        a = O.arms(img, p)
        H, W, _ = img.shape
        for y in range(H):
            for x in range(W):
                for e, (ex, ey) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
                    assert a[y, x, e] == brute_arm(img, x, y, ex, ey, p), (trial, y, x, e)


def test_arms_constant_image_reach_border_or_l1():
    H, W = 50, 90
    img = np.full((H, W, 3), 90, np.uint8)
    a = O.arms(img, P).astype(int)
    ys, xs = np.mgrid[0:H, 0:W]
    L1 = P.arm_l1
    assert (a[..., 0] == np.minimum(L1, xs)).all()
    assert (a[..., 1] == np.minimum(L1, W - 1 - xs)).all()
    assert (a[..., 2] == np.minimum(L1, ys)).all()
    assert (a[..., 3] == np.minimum(L1, H - 1 - ys)).all()


def test_arms_stop_at_stripe_edges():
    H, W, s = 9, 40, 5
    cols = (np.arange(W) // s) % 2 * 200
    img = np.repeat(np.repeat(cols[None, :, None], H, 0), 3, 2).astype(np.uint8)
    a = O.arms(img, P).astype(int)
    xs = np.arange(W)
    assert (a[:, :, 0] == (xs % s)[None]).all()
    assert (a[:, :, 1] == (s - 1 - xs % s)[None]).all()


def test_arms_second_threshold_applies_beyond_l2():
    # a slow ramp (step 1 per pixel): Dc(p_j, p) = j, so with tau2 = 6 the arm
    # can pass L2 only while j < 6; with L2 >= L1 the rule is single-threshold.
    W = 60
    v = np.clip(np.arange(W), 0, 255)
    img = grey_image(np.repeat(v[None, :], 3, 0))
    p = O.Params(arm_l1=30, arm_l2=3, tau1=20, tau2=6)
    a = O.arms(img, p)
    assert a[1, 0, 1] == 5            # j=4,5 beyond L2 pass (4,5 < 6), j=6 fails
    p2 = O.Params(arm_l1=30, arm_l2=30, tau1=20, tau2=6)
    assert O.arms(img, p2)[1, 0, 1] == 19   # tau1: Dc = j < 20


# ------------------------------------------------------------ Eq. 1 cost
def _eq1_exact(ad_sum, ham, lmin):
    """Eq. 1 evaluated symbolically at the Sect. 7.2 parameters (40 digits)."""
    g, e, lad, lc = sympy.Integer(1), sympy.Rational(4, 5), sympy.Integer(10), sympy.Integer(40)
    alpha = 1 - sympy.exp(-g / (lmin + e))
    c = alpha * (1 - sympy.exp(-sympy.Rational(ad_sum, 3) / lad)) + \
        (1 - alpha) * (1 - sympy.exp(-sympy.Integer(ham) / lc))
    return float(sympy.N(c, 40)), float(sympy.N(alpha, 40))


@pytest.mark.parametrize("ad,ham,lmin", [(0, 0, 0), (30, 0, 0), (0, 40, 34), (765, 62, 3),
                                         (1, 1, 17), (90, 13, 5)])
def test_eq1_closed_form_points(ad, ham, lmin):
    c, a = _eq1_exact(ad, ham, lmin)
    assert O.cost_terms(ad, ham, lmin) == pytest.approx(c, rel=1e-14, abs=1e-15)
    assert O.alpha(lmin) == pytest.approx(a, rel=1e-14)


def test_alpha_shrinks_as_arms_grow():
    # Sect. 4.2.1: a longer shortest arm means weaker texture and a smaller
    # weight on the AD measure.
    a = [O.alpha(l) for l in range(0, 35)]
    assert all(0.0 < x < 1.0 for x in a)
    assert all(a[i] > a[i + 1] for i in range(34))


def test_eq1_bounds_and_monotonicity():
    assert O.cost_terms(0, 0, 5) == 0.0
    assert O.cost_terms(765, 62, 0) < 1.0
    for lmin in (0, 4, 34):
        row = [O.cost_terms(ad, 7, lmin) for ad in range(0, 766, 15)]
        assert all(row[i] < row[i + 1] for i in range(len(row) - 1))
        col = [O.cost_terms(20, h, lmin) for h in range(63)]
        assert all(col[i] < col[i + 1] for i in range(62))


def test_eq1_weight_limits():
    # gamma_L -> large: alpha -> 1, only the AD term remains;
    # gamma_L -> 0: alpha -> 0, only the census term remains.
    big = O.Params(gamma_l=1e6)
    small = O.Params(gamma_l=1e-12)
    assert O.cost_terms(30, 50, 3, big) == pytest.approx(1 - np.exp(-1.0), rel=1e-9)
    assert O.cost_terms(30, 40, 3, small) == pytest.approx(1 - np.exp(-1.0), rel=1e-9)


# ----------------------------------------------------- Eq. 2 aggregation
def _region(arms_img, x, y):
    """N_p as an explicit coordinate set: for every q on p's vertical arm,
    the pixels of q's own horizontal segment."""
    l, r, u, d = (int(v) for v in arms_img[y, x])
    pts = set()
    for yy in range(y - u, y + d + 1):
        ql, qr = int(arms_img[yy, x, 0]), int(arms_img[yy, x, 1])
        for xx in range(x - ql, x + qr + 1):
            pts.add((xx, yy))
    return pts


def _raw_costs_left(left, right, D, p):
    H, W, _ = left.shape
    cl, cr = O.census(left), O.census(right)
    al = O.arms(left, p)
    lmin = al.min(axis=2)
    C = np.ones((D, H, W))
    li = left.astype(int)
    ri = right.astype(int)
    for d in range(D):
        for y in range(H):
            for x in range(d, W):
                ad = int(np.abs(li[y, x] - ri[y, x - d]).sum())
                ham = bin(int(cl[y, x]) ^ int(cr[y, x - d])).count("1")
                C[d, y, x] = O.cost_terms(ad, ham, int(lmin[y, x]), p)
    return C, al


def test_aggregation_equals_brute_force_region_mean():
    rng = np.random.default_rng(6)
    base = rng.integers(0, 256, (3, 4, 3))
    left = np.clip(np.kron(base, np.ones((4, 4, 1))) + rng.integers(-8, 9, (12, 16, 3)),
                   0, 255).astype(np.uint8)
    right = np.roll(left, -2, axis=1)
    right[:, -2:] = rng.integers(0, 256, (12, 2, 3))
    p = O.Params(arm_l1=5, arm_l2=2)
    D = 5
    res = O.match(left, right, D, p, volume=True)
    C, al = _raw_costs_left(left, right, D, p)
    for y in range(12):
        for x in range(16):
            pts = _region(al, x, y)
            for d in range(D):
                ref = sum(C[d, yy, xx] for xx, yy in pts) / len(pts)
                assert res.vol_l[d, y, x] == pytest.approx(ref, rel=1e-12, abs=1e-15)


def test_aggregation_box_special_case_matches_integral_image():
    # With no colour stop (tau = 256) and L2 = L1 = r, arms are the clipped
    # r-box, so Eq. 2 is a clipped box mean, computed here by cumulative sums.
    rng = np.random.default_rng(7)
    H, W, D, r = 20, 26, 4, 3
    left = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    right = rng.integers(0, 256, (H, W, 3), dtype=np.uint8)
    p = O.Params(arm_l1=r, arm_l2=r, tau1=256, tau2=256)
    res = O.match(left, right, D, p, volume=True)
    C, _ = _raw_costs_left(left, right, D, p)
    for d in range(D):
        S = np.zeros((H + 1, W + 1))
        S[1:, 1:] = C[d].cumsum(0).cumsum(1)
        for y in range(H):
            for x in range(W):
                y0, y1, x0, x1 = max(0, y - r), min(H, y + r + 1), max(0, x - r), min(W, x + r + 1)
                box = S[y1, x1] - S[y0, x1] - S[y1, x0] + S[y0, x0]
                n = (y1 - y0) * (x1 - x0)
                assert res.vol_l[d, y, x] == pytest.approx(box / n, rel=1e-12, abs=1e-14)


# ----------------------------------------------------------- Eq. 3 WTA
def test_identical_views_give_zero_disparity():
    rng = np.random.default_rng(8)
    img = scenes._texture(rng, 40, 48)
    img = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    res = O.match(img, img, 12)
    assert (res.disp_l == 0).all() and (res.disp_r == 0).all()
    assert (res.best_l == 0).all() and (res.best_r == 0).all()
    assert (res.disp == 0).all()


def test_all_tied_costs_take_the_smallest_disparity():
    img = np.full((16, 60, 3), 77, np.uint8)
    D = 6
    res = O.match(img, img, D, O.Params(arm_l1=3, arm_l2=3))
    # away from the left border every in-range candidate costs exactly 0
    assert (res.disp_l[:, 3 + D:] == 0).all()
    assert (res.best_l[:, 3 + D:] == 0).all() and (res.second_l[:, 3 + D:] == 0).all()


def _interior_mask(gt, occ, margin):
    H, W = gt.shape
    edge = np.zeros_like(occ)
    edge[:, 1:] |= gt[:, 1:] != gt[:, :-1]
    edge[1:, :] |= gt[1:, :] != gt[:-1, :]
    bad = edge | occ
    from scipy import ndimage
    near = ndimage.binary_dilation(bad, iterations=margin)
    m = ~near
    m[:margin] = m[-margin:] = False
    m[:, :margin] = m[:, -margin:] = False
    return m


def test_wta_recovers_ground_truth_in_textured_plane_interiors():
    s = scenes.config_scene(1)
    res = O.match(s.left, s.right, s.D)
    gt = np.rint(s.disp).astype(np.int16)
    m = _interior_mask(gt, s.occluded, P.arm_l1 + 4)
    assert m.sum() > 5000
    acc = (res.disp_l[m] == gt[m]).mean()
    assert acc >= 0.99, acc


# -------------------------------------------------------- LR check
def test_lr_check_hand_cases():
    dl = np.array([[0, 1, 2, 2, 5, 1]], np.int16)
    dr = np.array([[0, 3, 0, 9, 2, 4]], np.int16)
    # x=0: d=0 -> dr[0]=0 ok; x=1: d=1 -> dr[0]=0 |1-0|<=1 ok; x=2: d=2 -> dr[0]=0 bad;
    # x=3: d=2 -> dr[1]=3 ok; x=4: d=5 -> x-d<0 bad; x=5: d=1 -> dr[4]=2 ok
    assert O.lr_check(dl, dr, 1).tolist() == [[0, 1, -1, 2, -1, 1]]
    assert O.lr_check(dl, dr, 0).tolist() == [[0, -1, -1, -1, -1, -1]]
    assert O.lr_check(dl, dr, -1).tolist() == dl.tolist()


def test_mirror_swap_symmetry():
    # Swapping the views and mirroring both rows turns the right-reference
    # problem into the left-reference one: d_L' = mirror(d_R), d_R' = mirror(d_L).
    s = scenes.plane_scene(96, 40, 16, 4, seed=11, drange=(2, 12), noise_sigma=1.0)
    a = O.match(s.left, s.right, s.D)
    b = O.match(s.right[:, ::-1], s.left[:, ::-1], s.D)
    assert (b.disp_l == a.disp_r[:, ::-1]).all()
    assert (b.disp_r == a.disp_l[:, ::-1]).all()
    assert np.allclose(b.best_l, a.best_r[:, ::-1], rtol=1e-12, atol=0)
    assert (b.disp == O.lr_check(b.disp_l, b.disp_r, 1)).all()


def test_row_window_equals_full_run():
    s = scenes.config_scene(1)
    full = O.match(s.left, s.right, s.D)
    part = O.match(s.left, s.right, s.D, rows=(100, 140))
    assert (part.disp_l == full.disp_l[100:140]).all()
    assert (part.disp_r == full.disp_r[100:140]).all()
    assert (part.best_l == full.best_l[100:140]).all()


def test_arms_consecutive_colour_rule():
    # Each step differs from p by only 10 but from its predecessor by 20 at
    # j = 2: the neighbour-to-neighbour condition alone stops the arm there.
    row = np.array([100] + [110, 90] * 20, np.int64)
    img = grey_image(np.repeat(row[None, :], 3, 0).astype(np.uint8))
    a = O.arms(img, P)
    assert a[1, 0, 1] == 1
    # without the jump (110, 110, ...) only the L2/tau2 rule stops it
    row2 = np.array([100] + [110] * 40, np.int64)
    a2 = O.arms(grey_image(np.repeat(row2[None, :], 3, 0).astype(np.uint8)), P)
    assert a2[1, 0, 1] == P.arm_l2


def test_arms_brute_force_with_strong_noise():
    rng = np.random.default_rng(15)
    p = O.Params(arm_l1=6, arm_l2=2, tau1=20, tau2=9)
    base = rng.integers(0, 256, (3, 4, 3))
    img = np.kron(base, np.ones((4, 4, 1))).astype(np.int64)
    img = np.clip(img + rng.integers(-12, 13, img.shape), 0, 255).astype(np.uint8)
    a = O.arms(img, p)
    for y in range(img.shape[0]):
        for x in range(img.shape[1]):
            for e, (ex, ey) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1))):
                assert a[y, x, e] == brute_arm(img, x, y, ex, ey, p), (y, x, e)


# ----------------------------------------------------------------- Eq. 4 vote
def full_arms(H, W):
    """Arms reaching the image border in every direction: N_p = whole image."""
    a = np.zeros((H, W, 4), np.uint8)
    ys, xs = np.mgrid[0:H, 0:W]
    a[..., 0], a[..., 1], a[..., 2], a[..., 3] = xs, W - 1 - xs, ys, H - 1 - ys
    return a


def random_arms(rng, H, W, reach=3):
    """Arms within the image, at most `reach` long."""
    ys, xs = np.mgrid[0:H, 0:W]
    a = np.zeros((H, W, 4), np.uint8)
    for k, room in enumerate((xs, W - 1 - xs, ys, H - 1 - ys)):
        a[..., k] = np.minimum(room, rng.integers(0, reach + 1, (H, W)))
    return a


def vote_bruteforce(disp, arm, D, iters, d_min=0):
    """Eq. 4 written from the definition: the region as a set of coordinates
    (union over q on p's vertical arm of q's horizontal segment), a Python
    dictionary of counts, max count with the smallest d; d in [d_min, d_min + D)."""
    H, W = disp.shape
    cur = disp.astype(int).copy()
    for _ in range(iters):
        nxt = cur.copy()
        for y in range(H):
            for x in range(W):
                if not d_min <= cur[y, x] < d_min + D:
                    nxt[y, x] = -1
                    continue
                region = set()
                for yy in range(y - int(arm[y, x, 2]), y + int(arm[y, x, 3]) + 1):
                    l, r = int(arm[yy, x, 0]), int(arm[yy, x, 1])
                    region.update((xx, yy) for xx in range(x - l, x + r + 1))
                counts = {}
                for (xx, yy) in region:
                    v = cur[yy, xx]
                    if d_min <= v < d_min + D:
                        counts[v] = counts.get(v, 0) + 1
                top = max(counts.values())
                nxt[y, x] = min(v for v, c in counts.items() if c == top)
        cur = nxt
    return cur.astype(np.int16)


def test_vote_constant_map_is_a_fixed_point():
    s = scenes.plane_scene(40, 30, 16, 3, seed=11, drange=(1, 14))
    arm = O.arms(s.left)
    d = np.full((30, 40), 7, np.int16)
    d[::5, ::3] = -1
    for k in (1, 3):
        out = O.vote(d, arm, 16, k)
        assert np.array_equal(out, d)


def test_vote_replaces_an_isolated_outlier():
    d = np.full((9, 9), 4, np.int16)
    d[4, 4] = 9
    out = O.vote(d, full_arms(9, 9), 12, 1)
    assert (out == 4).all()


def test_vote_tie_takes_the_smallest_disparity():
    # two pixels joined by their arms, one vote each
    d = np.array([[5, 3]], np.int16)
    a = np.array([[[0, 1, 0, 0], [1, 0, 0, 0]]], np.uint8)
    assert O.vote(d, a, 8, 1).tolist() == [[3, 3]]


def test_vote_invalid_pixels_neither_vote_nor_change():
    d = np.array([[-1, -1, 2, -1, 7]], np.int16)
    out = O.vote(d, full_arms(1, 5), 8, 1)
    assert out.tolist() == [[-1, -1, 2, -1, 2]]   # {2: 1, 7: 1}: tie -> 2
    d2 = np.array([[-1, 6, -1]], np.int16)
    assert O.vote(d2, full_arms(1, 3), 8, 2).tolist() == [[-1, 6, -1]]
    # values beyond the range are invalid too: no vote, written as -1
    d3 = np.array([[9, 4, 4, 12]], np.int16)
    assert O.vote(d3, full_arms(1, 4), 8, 1).tolist() == [[-1, 4, 4, -1]]


def test_vote_region_is_h_then_v():
    # p's vertical arm reaches row 0, whose horizontal arm reaches x = 0;
    # row 1's horizontal arm is empty, so x = 0 of row 1 is not in N_p
    d = np.array([[3, 5], [3, 5]], np.int16)
    a = np.zeros((2, 2, 4), np.uint8)
    a[1, 1, 2] = 1         # (1, 1): up arm 1
    a[0, 1, 0] = 1         # (0, 1): left arm 1
    out = O.vote(d, a, 8, 1)
    # N_(1,1) = {(1,1), (1,0), (0,0)} in (x, y): votes 5, 5, 3 -> 5
    assert out[1, 1] == 5
    a[1, 1, 0] = 1         # now row 1 also reaches x = 0: votes 5, 3, 5, 3 -> tie -> 3
    assert O.vote(d, a, 8, 1)[1, 1] == 3


def test_vote_matches_bruteforce():
    rng = np.random.default_rng(4)
    for H, W, D in ((5, 7, 6), (8, 6, 4), (1, 9, 5)):
        d = rng.integers(-1, D + 1, (H, W)).astype(np.int16)   # D: out of range
        a = random_arms(rng, H, W)
        for k in (1, 2, 3):
            assert np.array_equal(O.vote(d, a, D, k), vote_bruteforce(d, a, D, k)), (H, W, D, k)


def test_vote_with_d_min_matches_bruteforce():
    # Eq. 4's range [d_min, d_max]: values below d_min are invalid like -1
    rng = np.random.default_rng(14)
    for H, W, D, dmin in ((5, 7, 6, 3), (8, 6, 4, 9), (1, 9, 5, 1)):
        d = rng.integers(-1, dmin + D + 1, (H, W)).astype(np.int16)
        a = random_arms(rng, H, W)
        for k in (1, 2):
            got = O.vote(d, a, D, k, d_min=dmin)
            assert np.array_equal(got, vote_bruteforce(d, a, D, k, d_min=dmin)), (H, W, D, dmin, k)
            assert ((got == -1) | ((got >= dmin) & (got < dmin + D))).all()


def test_vote_iterations_compose():
    rng = np.random.default_rng(5)
    d = rng.integers(-1, 12, (20, 24)).astype(np.int16)
    a = random_arms(rng, 20, 24, reach=5)
    once = O.vote(d, a, 12, 1)
    assert np.array_equal(O.vote(d, a, 12, 2), O.vote(once, a, 12, 1))
    assert np.array_equal(O.vote(d, a, 12, 0), d)


# ----------------------------------------------------------------- quarter size + depth
def test_downscale_inverts_block_replication():
    rng = np.random.default_rng(12)
    small = rng.integers(0, 256, (13, 17, 3), dtype=np.uint8)
    big = np.repeat(np.repeat(small, 2, axis=0), 2, axis=1)
    assert np.array_equal(O.downscale(big), small)
    # an odd last row and column are dropped
    odd = np.concatenate([big, rng.integers(0, 256, (1, 34, 3), dtype=np.uint8)], axis=0)
    odd = np.concatenate([odd, rng.integers(0, 256, (27, 1, 3), dtype=np.uint8)], axis=1)
    assert np.array_equal(O.downscale(odd), small)


def test_downscale_rounds_the_block_mean_half_up():
    rng = np.random.default_rng(13)
    img = rng.integers(0, 256, (2, 2 * 500, 3), dtype=np.uint8)
    out = O.downscale(img)
    for x in range(500):
        for c in range(3):
            vals = [int(img[0, 2 * x, c]), int(img[0, 2 * x + 1, c]), int(img[1, 2 * x, c]), int(img[1, 2 * x + 1, c])]
            mean = sum(vals) / 4.0
            assert out[0, x, c] == int(np.floor(mean + 0.5)), (vals, out[0, x, c])


def test_depth_closed_forms_and_missing():
    d = np.array([[2, 0, -1], [4, 1, 7]], np.int16)
    z = O.depth(d, 7, 5, 700.0, 0.1)
    assert z.shape == (5, 7)
    assert z[0, 0] == z[1, 1] == 700.0 * 0.1 / 4          # d = 2 -> 2d = 4 at full size
    assert z[2, 0] == z[3, 1] == 700.0 * 0.1 / 8
    assert z[2, 2] == 700.0 * 0.1 / 2 and z[3, 5] == 700.0 * 0.1 / 14
    assert (z[0:2, 2:6] == 0).all()                       # d = 0 and d = -1: missing
    assert (z[4, :] == 0).all() and (z[:, 6] == 0).all()  # odd last row / column
    v = np.repeat(np.repeat(d, 2, axis=0), 2, axis=1)
    ok = v > 0
    assert np.allclose(z[:4, :6][ok] * 2 * v[ok], 70.0, rtol=1e-15)   # Z * (2d) = f B


def test_quarter_size_path_recovers_a_plane_depth():
    # a fronto-parallel textured plane at full-size disparity 2*d0: matched at
    # half size it is found at d0, so its depth is f B / (2 d0)
    d0, f, B = 6, 800.0, 0.12
    s = scenes.plane_scene(128, 96, 16, 0, seed=31, drange=(2 * d0, 2 * d0))
    assert np.allclose(s.disp[:, 2 * d0 + 8:], 2 * d0)
    Lh, Rh = O.downscale(s.left), O.downscale(s.right)
    m = O.match(Lh, Rh, 12)
    z = O.depth(m.disp, 128, 96, f, B)
    interior = z[8:-8, 2 * (d0 + 8):-8]
    assert (interior == f * B / (2 * d0)).mean() > 0.95


# ----------------------------------------------------------------- arm smoothing (Sect. 4.1)
def test_arm_smoothing_is_the_library_grey_opening():
    from scipy import ndimage
    rng = np.random.default_rng(21)
    for H, W in ((1, 1), (2, 7), (17, 23)):
        a = rng.integers(0, 35, (H, W, 4)).astype(np.uint8)
        want = np.stack([ndimage.grey_opening(a[..., k], size=(3, 3), mode="nearest") for k in range(4)], axis=-1)
        assert np.array_equal(O.arms_smooth(a), want), (H, W)


def test_arm_smoothing_is_an_opening():
    s = scenes.plane_scene(60, 40, 16, 4, seed=22, drange=(1, 14), noise_sigma=3.0)
    a = O.arms(s.left)
    o = O.arms_smooth(a)
    assert (o <= a).all()                                  # anti-extensive
    assert np.array_equal(O.arms_smooth(o), o)             # idempotent
    assert np.array_equal(O.arms(s.left, O.Params(smooth_arms=1)), o)
    ys, xs = np.mgrid[0:40, 0:60]
    room = np.stack([xs, 59 - xs, ys, 39 - ys], axis=-1)
    assert (o <= room).all()                               # still inside the image


def test_arm_smoothing_removes_spikes_keeps_plateaus():
    a = np.full((9, 9, 4), 2, np.uint8)
    a[1, 1, 0] = 30                 # isolated long arm: gone
    a[4:7, 4:7, 1] = 20             # 3x3 plateau: kept
    o = O.arms_smooth(a)
    assert o[1, 1, 0] == 2
    assert (o[4:7, 4:7, 1] == 20).all() and (o[..., 1].sum() - 9 * 20) == (81 - 9) * 2


def test_match_with_smoothing_aggregates_over_the_opened_arms():
    # the region mean of Eq. 2 by explicit coordinate sets, with L_min and the
    # regions taken from the opened arms (the opening itself is pinned above)
    rng = np.random.default_rng(24)
    base = rng.integers(0, 256, (3, 4, 3))
    left = np.clip(np.kron(base, np.ones((4, 4, 1))) + rng.integers(-8, 9, (12, 16, 3)), 0, 255).astype(np.uint8)
    right = np.roll(left, -2, axis=1)
    p = O.Params(arm_l1=5, arm_l2=2, smooth_arms=1)
    res = O.match(left, right, 5, p, volume=True)
    C, al = _raw_costs_left(left, right, 5, p)
    assert np.array_equal(al, O.arms_smooth(O.arms(left, O.Params(arm_l1=5, arm_l2=2))))
    assert not np.array_equal(al, O.arms(left, O.Params(arm_l1=5, arm_l2=2)))
    for y in range(12):
        for x in range(16):
            pts = _region(al, x, y)
            for d in range(5):
                ref = sum(C[d, yy, xx] for xx, yy in pts) / len(pts)
                assert res.vol_l[d, y, x] == pytest.approx(ref, rel=1e-12, abs=1e-15)


# ----------------------------------------------------------------- densification (Sect. 6)
from oracle import densify as DN   # noqa: E402


def _dn_inputs(rng, H, W, frac=0.1, contour=False):
    ds = np.where(rng.random((H, W)) < frac, rng.uniform(0.5, 5.0, (H, W)), 0.0)
    B = (rng.random((H, W)) < 0.15).astype(np.uint8) if contour else np.zeros((H, W), np.uint8)
    return ds, B, rng.random((H, W)), rng.random((H, W))


def test_densify_pair_weight_cases():
    assert DN.pair_weight(1, 0, 0.1, 0.2) == 0.0 and DN.pair_weight(0, 1, 0.0, 0.0) == 0.0   # Eq. 16 first case
    assert DN.pair_weight(1, 1, 0.3, 0.6) == pytest.approx(0.7)
    assert DN.pair_weight(0, 0, 0.3, 0.6) == pytest.approx(0.7)
    assert DN.pair_weight(0, 0, 1.5, 2.0) == 0.0                                            # max(., 0)


def test_densify_without_smoothness_is_the_weighted_data_mean():
    rng = np.random.default_rng(41)
    ds, B, mf, mi = _dn_inputs(rng, 6, 7, 0.5)
    dp = np.where(rng.random((6, 7)) < 0.5, rng.uniform(1, 3, (6, 7)), 0.0)
    p = DN.DenseParams(lambda_d=0.8, lambda_s=0.0, lambda_s2=0.3)
    D = DN.densify(ds, B, mf, mi, dp, p)
    ws, wt = (ds > 0) * 0.8, (dp > 0) * 0.3
    want = np.where(ws + wt > 0, (ws * ds + wt * dp) / np.where(ws + wt > 0, ws + wt, 1), 0.0)
    assert np.allclose(D, want, rtol=1e-12, atol=1e-14)


def test_densify_single_anchor_spreads_a_constant():
    ds = np.zeros((9, 11)); ds[4, 5] = 2.5
    z = np.zeros((9, 11))
    D = DN.densify(ds, z.astype(np.uint8), z, z)
    assert np.allclose(D, 2.5, rtol=1e-12)


def test_densify_contour_splits_and_undetermined_is_missing():
    ds = np.zeros((6, 10)); ds[2, 1] = 1.0; ds[3, 8] = 4.0
    B = np.zeros((6, 10), np.uint8); B[:, 5:] = 1          # w = 0 across x = 4 | 5
    z = np.zeros((6, 10))
    D = DN.densify(ds, B, z, z)
    assert np.allclose(D[:, :5], 1.0) and np.allclose(D[:, 5:], 4.0)
    # pixels cut off from every anchor stay 0: with s = 1 on x >= 5, pairs
    # inside that band get w = 0 (Eq. 16), while the pairs x = 4 | 5 keep
    # w = 1 - min(0, 1) = 1, so column 5 joins the anchored left part
    s = np.zeros((6, 10)); s[:, 5:] = 1.0
    D2 = DN.densify(np.where(np.arange(10) < 5, ds, 0.0), np.zeros((6, 10), np.uint8), s, np.ones((6, 10)))
    assert np.allclose(D2[:, :6], 1.0) and (D2[:, 6:] == 0).all()


def test_densify_minimises_the_energy_of_eq20():
    rng = np.random.default_rng(42)
    ds, B, mf, mi = _dn_inputs(rng, 7, 8, 0.2, contour=True)
    dp = np.where(rng.random((7, 8)) < 0.2, rng.uniform(1, 3, (7, 8)), 0.0)
    D = DN.densify(ds, B, mf, mi, dp)
    e0 = DN.energy(D, ds, B, mf, mi, dp)
    det = D != 0
    for k in range(20):
        v = rng.standard_normal(D.shape) * det
        for eps in (1e-3, -1e-3):
            assert DN.energy(D + eps * v, ds, B, mf, mi, dp) > e0
        # zero directional derivative (central difference of a quadratic is exact)
        g = (DN.energy(D + 1e-3 * v, ds, B, mf, mi, dp) - DN.energy(D - 1e-3 * v, ds, B, mf, mi, dp)) / 2e-3
        assert abs(g) < 1e-7 * max(1.0, e0)


# ----------------------------------------------------------------- aggregation order variant
def _region_vh(arms_img, x, y):
    """The other order as a coordinate set: for every q on p's horizontal arm,
    the pixels of q's own vertical segment."""
    l, r = int(arms_img[y, x, 0]), int(arms_img[y, x, 1])
    pts = set()
    for xx in range(x - l, x + r + 1):
        qu, qd = int(arms_img[y, xx, 2]), int(arms_img[y, xx, 3])
        for yy in range(y - qu, y + qd + 1):
            pts.add((xx, yy))
    return pts


def test_v_then_h_aggregation_equals_brute_force_region_mean():
    rng = np.random.default_rng(61)
    base = rng.integers(0, 256, (3, 4, 3))
    left = np.clip(np.kron(base, np.ones((4, 4, 1))) + rng.integers(-8, 9, (12, 16, 3)), 0, 255).astype(np.uint8)
    right = np.roll(left, -2, axis=1)
    right[:, -2:] = rng.integers(0, 256, (12, 2, 3))
    p = O.Params(arm_l1=5, arm_l2=2, agg_order=1)
    res = O.match(left, right, 5, p, volume=True)
    C, al = _raw_costs_left(left, right, 5, p)
    differs = False
    for y in range(12):
        for x in range(16):
            pts = _region_vh(al, x, y)
            differs |= pts != _region(al, x, y)
            for d in range(5):
                ref = sum(C[d, yy, xx] for xx, yy in pts) / len(pts)
                assert res.vol_l[d, y, x] == pytest.approx(ref, rel=1e-12, abs=1e-15)
    assert differs   # the two orders give different regions on this input


def test_aggregation_orders_agree_on_box_arms():
    # no colour stop and L2 = L1: every arm is the clipped box radius, so both
    # orders cover the same clipped box
    rng = np.random.default_rng(62)
    left = rng.integers(0, 256, (14, 19, 3), dtype=np.uint8)
    right = rng.integers(0, 256, (14, 19, 3), dtype=np.uint8)
    kw = dict(arm_l1=3, arm_l2=3, tau1=256, tau2=256)
    a = O.match(left, right, 4, O.Params(**kw), volume=True)
    b = O.match(left, right, 4, O.Params(agg_order=1, **kw), volume=True)
    assert np.allclose(a.vol_l, b.vol_l, rtol=1e-12, atol=1e-15)
    assert np.array_equal(a.disp_l, b.disp_l) and np.array_equal(a.disp, b.disp)


# ------------------------------------------- decision in the kernel's precision
# The argmin of Eq. 3 is decided by floating point and the paper fixes no
# precision, so the GPU's maps are compared with the oracle's decision taken
# in the kernel's precision (FP32 Eq. 1, fixed point, exact integer sums).
# That path is pinned to the FP64 oracle: every pixel where the two decisions
# differ must have FP64 best and second-best within twice the error bound of
# the kernel's cost evaluation, and such pixels are rare.  A wrong table index, weight or sum order would
# move whole regions off the FP64 minimum and fail here.
@pytest.mark.parametrize("case", ["fine", "mixed", "mixed_vh", "mixed_smooth", "params"])
def test_kernel_precision_decision_differs_from_fp64_only_at_near_ties(case):
    texture = "fine" if case == "fine" else "mixed"
    s = scenes.plane_scene(120, 72, 24, 5, seed=scenes.seed_for(2, 970), slanted=True, noise_sigma=2.0,
                           drange=(2, 21), texture=texture)
    p = {"fine": O.Params(), "mixed": O.Params(), "mixed_vh": O.Params(agg_order=1),
         "mixed_smooth": O.Params(smooth_arms=1),
         "params": O.Params(lambda_ad=30.0, lambda_census=15.0, gamma_l=3.0, eps=0.5, arm_l1=9, arm_l2=4)}[case]
    r = O.match(s.left, s.right, s.D, p, quantized=True)
    total = 0
    for q, d, b, sc in ((r.qdisp_l, r.disp_l, r.best_l, r.second_l), (r.qdisp_r, r.disp_r, r.best_r, r.second_r)):
        # the kernel's aggregated cost is within 1e-6 of the FP64 one (0.5/S
        # of rounding plus a few FP32 ulp per term, any L1 <= 40): a flip
        # needs a gap of at most twice that
        near = (sc - b) <= 2 * 1.0e-6
        diff = q != d
        assert not (diff & ~near).any(), f"{int((diff & ~near).sum())} decisions differ beyond the bound"
        total += int(diff.sum())
    assert total <= 0.001 * 2 * s.W * s.H
    assert np.array_equal(r.qdisp, O.lr_check(r.qdisp_l, r.qdisp_r, p.lr_tol))


def test_kernel_precision_decision_on_identical_views_and_rows():
    # identical views: every cost at d = 0 is exactly 0 in both precisions
    rng = np.random.default_rng(5)
    img = np.clip(np.rint(scenes._texture(rng, 30, 40)), 0, 255).astype(np.uint8)
    r = O.match(img, img, 8, quantized=True)
    assert (r.qdisp_l == 0).all() and (r.qdisp_r == 0).all()
    # a row band equals the same rows of the full run (the decision is local)
    s = scenes.plane_scene(64, 48, 12, 3, seed=scenes.seed_for(2, 971), drange=(2, 9), texture="mixed")
    full = O.match(s.left, s.right, s.D, quantized=True)
    part = O.match(s.left, s.right, s.D, rows=(20, 30), quantized=True)
    assert np.array_equal(part.qdisp_l, full.qdisp_l[20:30]) and np.array_equal(part.qdisp_r, full.qdisp_r[20:30])


def test_kernel_precision_decision_catches_a_planted_cost_error():
    # the same pin with the oracle's own FP64 decision perturbed stands in
    # for a broken kernel-precision path: shifting one view's costs by a
    # constant per d (a dropped term) must trip the near-tie rule
    s = scenes.plane_scene(96, 64, 16, 4, seed=scenes.seed_for(2, 972), drange=(2, 13), texture="mixed")
    r = O.match(s.left, s.right, s.D, quantized=True, volume=True)
    bent = np.argmin(r.vol_l + 0.02 * np.arange(s.D)[:, None, None], axis=0).astype(np.int16)
    near = (r.second_l - r.best_l) <= 1e-4 * r.best_l + 1e-6
    assert ((bent != r.disp_l) & ~near).any()


# ----------------------------------------------------------------- Eq. 3 range [d_min, d_max]
@pytest.mark.parametrize("order", [0, 1])
def test_d_min_search_is_the_sub_range_of_the_full_search(order):
    # Eqs. 2-3 with d in [k, k + D): the aggregated costs are planes k .. k + D - 1
    # of the search from 0 (Eq. 2 does not depend on the range), the decision
    # the first argmin over those planes only, the checked map the LR check of
    # the two absolute maps
    s = scenes.plane_scene(48, 20, 24, 3, seed=21, drange=(6, 20), noise_sigma=2.0)
    k, D = 5, 14
    full = O.match(s.left, s.right, k + D, O.Params(agg_order=order), volume=True)
    sub = O.match(s.left, s.right, D, O.Params(agg_order=order, d_min=k), volume=True, quantized=True)
    for v, (fv, sv, sd, sb) in enumerate(((full.vol_l, sub.vol_l, sub.disp_l, sub.best_l),
                                          (full.vol_r, sub.vol_r, sub.disp_r, sub.best_r))):
        np.testing.assert_array_equal(sv, fv[k:])
        assert np.array_equal(sd, k + np.argmin(fv[k:], axis=0)), v
        np.testing.assert_array_equal(sb, fv[k:].min(axis=0))
        assert (sd >= k).all() and (sd < k + D).all()
    assert np.array_equal(sub.disp, O.lr_check(sub.disp_l, sub.disp_r, P.lr_tol))
    assert (sub.qdisp_l >= k).all() and (sub.qdisp_r < k + D).all()
    # a range that holds the whole truth gives the same map as the full search
    # wherever the full search's decision lies inside it
    inside = (full.disp_l >= k) & (full.disp_l < k + D)
    assert inside.mean() > 0.8
    assert np.array_equal(sub.disp_l[inside], full.disp_l[inside])
