"""Fixtures of tests/golden (written by tests/golden/make_golden.py):

- Eq. 1 at the Sect. 7.2 parameters, evaluated from the paper's formula at
  50 digits with mpmath (independent of the oracle): the oracle's cost terms
  must agree to FP64 round-off;
- a 16x12, D = 4 pair with the oracle's result stored: the oracle must
  reproduce it (regression), and the GPU must match it under the parity
  rule."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from tests import parity

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _eq1_rows():
    rows = []
    for line in open(os.path.join(HERE, "eq1_sect72.txt")):
        if line.startswith("#"):
            continue
        k, h, lmin, c = line.split()
        rows.append((int(k), int(h), int(lmin), float(c)))
    return rows


def _match_fixture():
    data = {}
    for line in open(os.path.join(HERE, "match_16x12_D4.txt")):
        if line.startswith("#"):
            continue
        parts = line.split()
        name, y, vals = parts[0], int(parts[1]), parts[2:]
        data.setdefault(name, {})[y] = vals
    out = {}
    for name, rows in data.items():
        a = [rows[y] for y in range(len(rows))]
        if name in ("left", "right"):
            out[name] = np.array(a, np.uint8).reshape(12, 16, 3)
        elif name in ("best_l", "second_l"):
            out[name] = np.array(a, np.float64)
        else:
            out[name] = np.array(a, np.int16)
    return out


def test_oracle_eq1_equals_50_digit_values():
    rows = _eq1_rows()
    assert len(rows) == 9 * 6 * 5
    p = O.Params()   # Sect. 7.2 values
    for k, h, lmin, c in rows:
        assert O.cost_terms(k, h, lmin, p) == pytest.approx(c, rel=1e-14, abs=1e-16), (k, h, lmin)


def test_oracle_reproduces_the_stored_match():
    f = _match_fixture()
    r = O.match(f["left"], f["right"], 4)
    for name in ("disp_l", "disp_r", "disp"):
        assert np.array_equal(getattr(r, name), f[name]), name
    assert np.allclose(r.best_l, f["best_l"], rtol=1e-12, atol=0)
    assert np.allclose(r.second_l, f["second_l"], rtol=1e-12, atol=0)


@pytest.mark.gpu
def test_gpu_matches_the_stored_match():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_02300_gb300 import binding
    f = _match_fixture()
    with binding.Stereo(0) as st:
        out, dl, dr, cl, cr = st.match_views(torch.from_numpy(f["left"]).cuda(), torch.from_numpy(f["right"]).cuda(), 4)
        torch.cuda.synchronize()
    dl = dl.cpu().numpy()
    parity.check_disparity(dl, f["disp_l"], f["best_l"], f["second_l"], "left disparity")
    parity.check_cost(cl.cpu().numpy(), f["best_l"], dl, f["disp_l"], "left cost")
    assert np.array_equal(out.cpu().numpy(), O.lr_check(dl, dr.cpu().numpy(), 1))
