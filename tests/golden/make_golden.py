"""Writes the fixtures of this folder.  Run from the repository root:

    python tests/golden/make_golden.py

eq1_sect72.txt   Eq. 1 (Sect. 4.2.1) at the parameters of Sect. 7.2
                 (lambda_AD = 10, lambda_census = 40, gamma_L = 1, eps = 0.8)
                 for a grid of channel sums k, Hamming distances h and
                 shortest arms L_min, evaluated from the paper's formula at
                 50 significant digits with mpmath (no oracle code):
                 C = alpha (1 - e^(-(k/3)/lambda_AD)) + (1 - alpha)(1 - e^(-h/lambda_census)),
                 alpha = 1 - e^(-gamma_L / (L_min + eps)), C_AD = k / 3 (the
                 mean of the three channel differences).
match_16x12_D4.txt  a seeded 16x12 pair and the oracle's result on it (left
                 and right disparities, consistency map, best and
                 second-best aggregated costs of the left view): written by
                 the oracle, a regression fixture for the GPU path.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def eq1():
    import mpmath as mp
    mp.mp.dps = 50
    lam_ad, lam_c, gam, eps = mp.mpf(10), mp.mpf(40), mp.mpf(1), mp.mpf("0.8")
    lines = ["# k h lmin C  (Eq. 1 at Sect. 7.2 parameters, 50-digit evaluation)"]
    for k in (0, 1, 2, 3, 30, 100, 255, 500, 765):
        for h in (0, 1, 7, 20, 40, 62):
            for lmin in (0, 1, 4, 17, 34):
                alpha = 1 - mp.e ** (-gam / (lmin + eps))
                c = alpha * (1 - mp.e ** (-(mp.mpf(k) / 3) / lam_ad)) + (1 - alpha) * (1 - mp.e ** (-mp.mpf(h) / lam_c))
                lines.append(f"{k} {h} {lmin} {mp.nstr(c, 30)}")
    with open(os.path.join(HERE, "eq1_sect72.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def match_fixture():
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import oracle as O
    rng = np.random.default_rng(2203)
    base = rng.integers(0, 256, (3, 4, 3))
    left = np.clip(np.kron(base, np.ones((4, 4, 1))) + rng.integers(-10, 11, (12, 16, 3)), 0, 255).astype(np.uint8)
    right = np.roll(left, -2, axis=1)
    right[:, -2:] = rng.integers(0, 256, (12, 2, 3))
    r = O.match(left, right, 4)
    lines = ["# 16x12 pair, D = 4: left, right (rgb rows), oracle disp_l, disp_r, disp, best_l, second_l"]
    for name, a in (("left", left), ("right", right)):
        for y in range(12):
            lines.append(f"{name} {y} " + " ".join(str(int(v)) for v in a[y].ravel()))
    for name, a in (("disp_l", r.disp_l), ("disp_r", r.disp_r), ("disp", r.disp)):
        for y in range(12):
            lines.append(f"{name} {y} " + " ".join(str(int(v)) for v in a[y]))
    for name, a in (("best_l", r.best_l), ("second_l", r.second_l)):
        for y in range(12):
            lines.append(f"{name} {y} " + " ".join(repr(float(v)) for v in a[y]))
    with open(os.path.join(HERE, "match_16x12_D4.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    eq1()
    match_fixture()
