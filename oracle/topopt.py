"""Density filter and optimality-criteria (OC) update (oracle, test only).

Neither is the paper's (it uses MMA, Sec. 2.3, and no filter is stated); both
are the textbook SIMP harness used to drive repeated solves:

* Density filter: x~_e = sum_j w_ej x_j / sum_j w_ej with hat weights
  w_ej = max(0, r - dist(e, j)) between element centroids (in element units),
  truncated at the domain boundary.  Its transpose maps dc/dx~ to dc/dx.
* OC: x_new = clip(x * (-dc / (lambda dv))^eta, x - move, x + move) within
  [0, 1]; lambda by bisection so that the filtered volume fraction hits V*.

Pinned by tests/test_oracle_topopt.py: the filter against a brute-force
loop over element pairs on tiny grids (plus row sums, identity at radius
<= 1, transpose); the OC step against its closed form on uniform
sensitivities, its box and move limits, the volume it reaches and the
optimality form shared by all unclipped elements.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def filter_matrix(N: int, rmin: float) -> sp.csr_matrix:
    """Row-normalised hat-weight filter H (M x M) on an N^3 element grid."""
    M = N ** 3
    R = int(np.ceil(rmin)) - 1 if float(rmin).is_integer() else int(np.floor(rmin))
    ez, ey, ex = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
    rows, cols, vals = [], [], []
    for dz in range(-R, R + 1):
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                w = rmin - np.sqrt(dx * dx + dy * dy + dz * dz)
                if w <= 0:
                    continue
                jx, jy, jz = ex + dx, ey + dy, ez + dz
                ok = (jx >= 0) & (jx < N) & (jy >= 0) & (jy < N) & (jz >= 0) & (jz < N)
                e = np.flatnonzero(ok)
                rows.append(e)
                cols.append(jx[ok] + N * (jy[ok] + N * jz[ok]))
                vals.append(np.full(e.size, w))
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(M, M))
    s = np.asarray(H.sum(axis=1)).ravel()
    return (sp.diags(1.0 / s) @ H).tocsr()


def oc_update(x, dc, dv, volfrac, H=None, move=0.2, eta=0.5,
              l1=0.0, l2=1e9, tol=1e-3):
    """One OC step; returns the new design x (the volume of H x_new ~= V*)."""
    x = np.asarray(x, float)
    dc = np.minimum(np.asarray(dc, float), -1e-300)
    while (l2 - l1) / (l1 + l2) > tol:
        lmid = 0.5 * (l1 + l2)
        xn = x * (-dc / (dv * lmid)) ** eta
        xn = np.clip(xn, np.maximum(0.0, x - move), np.minimum(1.0, x + move))
        vol = (H @ xn).mean() if H is not None else xn.mean()
        if vol > volfrac:
            l1 = lmid
        else:
            l2 = lmid
    return xn
