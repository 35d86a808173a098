"""FP64 oracle of the depth densification (Sect. 6, Eqs. 13-20).

TEST INFRASTRUCTURE ONLY: nothing in the product path imports this module;
the tests, the smoke check and the benchmark's CPU baseline do.

The dense map D minimises (Eq. 20)

    lambda_d  sum_p w_sparse(p) (D(p) - D_sparse(p))^2            (Eqs. 13, 14)
  + lambda_s  sum_p sum_{q in N4(p)} w_pq (D(p) - D(q))^2          (Eqs. 15-17)
  + lambda_s2 sum_p w_stable(p) (D(p) - D_pre(p))^2                (Eqs. 18, 19)

with w_sparse = [D_sparse > 0], w_stable = [D_pre > 0],
w_pq = 0 if exactly one of p, q lies on the depth contour B_dp, else
max(1 - min(s_p, s_q), 0), s = M_fuse * M_I.  Readings of what the paper
leaves open: N4 is cut at the image border; the double sum counts every
neighbour pair twice, as written; a pixel whose component of the w_pq > 0
graph holds no data or stability term is not determined by Eq. 20 and is
returned as 0 (missing).

Setting the gradient to zero gives the sparse symmetric system
  (lambda_d w_sparse + lambda_s2 w_stable) D(p) + 2 lambda_s sum_q w_pq (D(p) - D(q))
      = lambda_d w_sparse D_sparse(p) + lambda_s2 w_stable D_pre(p),
assembled here entry by entry and solved with scipy's sparse direct solver.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class DenseParams:
    lambda_d: float = 0.80    # Sect. 7.2
    lambda_s: float = 1.20    # Sect. 7.2
    lambda_s2: float = 0.02   # Sect. 7.2


def pair_weight(b_p, b_q, s_p, s_q):
    """Eq. 16: w_pq."""
    if int(b_p) + int(b_q) == 1:
        return 0.0
    return max(1.0 - min(float(s_p), float(s_q)), 0.0)


def system(d_sparse, contour, m_fuse, m_int, d_pre=None, p: DenseParams = DenseParams()):
    """(A, b) of the normal equations of Eq. 20 (scipy CSR, FP64), pixels in
    row-major order."""
    import scipy.sparse as sp
    H, W = d_sparse.shape
    n = H * W
    ds = np.asarray(d_sparse, np.float64).ravel()
    dp = np.zeros(n) if d_pre is None else np.asarray(d_pre, np.float64).ravel()
    B = np.asarray(contour).ravel()
    s = (np.asarray(m_fuse, np.float64) * np.asarray(m_int, np.float64)).ravel()   # Eq. 17
    w_sp = (ds > 0).astype(np.float64)   # Eq. 14
    w_st = (dp > 0).astype(np.float64)   # Eq. 19
    diag = p.lambda_d * w_sp + p.lambda_s2 * w_st
    b = p.lambda_d * w_sp * ds + p.lambda_s2 * w_st * dp
    rows, cols, vals = [], [], []
    for y in range(H):
        for x in range(W):
            i = y * W + x
            for (xx, yy) in ((x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)):
                if not (0 <= xx < W and 0 <= yy < H):
                    continue
                j = yy * W + xx
                w = pair_weight(B[i], B[j], s[i], s[j])
                if w == 0.0:
                    continue
                diag[i] += 2.0 * p.lambda_s * w
                rows.append(i); cols.append(j); vals.append(-2.0 * p.lambda_s * w)
    rows += list(range(n)); cols += list(range(n)); vals += list(diag)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    return A, b


def densify(d_sparse, contour, m_fuse, m_int, d_pre=None, p: DenseParams = DenseParams()) -> np.ndarray:
    """The minimiser of Eq. 20 (H, W) float64; 0 on undetermined components."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    from scipy.sparse.csgraph import connected_components
    H, W = d_sparse.shape
    A, b = system(d_sparse, contour, m_fuse, m_int, d_pre, p)
    n = H * W
    off = A - sp.diags(A.diagonal())
    ncomp, label = connected_components(off != 0, directed=False)
    anchored = np.zeros(ncomp, bool)
    data = np.asarray(d_sparse).ravel() > 0
    if d_pre is not None:
        data |= np.asarray(d_pre).ravel() > 0
    anchored[np.unique(label[data])] = True
    keep = anchored[label]
    x = np.zeros(n)
    if keep.any():
        idx = np.nonzero(keep)[0]
        x[idx] = spla.spsolve(A[idx][:, idx].tocsc(), b[idx])
    return x.reshape(H, W)


def energy(D, d_sparse, contour, m_fuse, m_int, d_pre=None, p: DenseParams = DenseParams()) -> float:
    """Eq. 20 evaluated term by term (loops over pixels and their N4)."""
    H, W = D.shape
    s = np.asarray(m_fuse, np.float64) * np.asarray(m_int, np.float64)
    e = 0.0
    for y in range(H):
        for x in range(W):
            if d_sparse[y, x] > 0:
                e += p.lambda_d * (D[y, x] - d_sparse[y, x]) ** 2
            if d_pre is not None and d_pre[y, x] > 0:
                e += p.lambda_s2 * (D[y, x] - d_pre[y, x]) ** 2
            for (xx, yy) in ((x - 1, y), (x + 1, y), (x, y - 1), (x, y + 1)):
                if 0 <= xx < W and 0 <= yy < H:
                    w = pair_weight(contour[y, x], contour[yy, xx], s[y, x], s[yy, xx])
                    e += p.lambda_s * w * (D[y, x] - D[yy, xx]) ** 2
    return e
