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


def _axis_weights_cells(N: int, r: int):
    """Per fine cell i of an axis refined r times: the coarse cells i0, i1 and the
    weight t of i1 for linear interpolation between coarse cell centres (fine
    centre at (i + 1/2)/r - 1/2 in coarse-centre units), constant beyond the
    outer centres."""
    i = np.arange(N * r)
    s = (i + 0.5) / r - 0.5
    i0 = np.floor(s).astype(np.int64)
    t = s - i0
    lo = i0 < 0
    hi = i0 >= N - 1
    i0 = np.where(lo, 0, np.where(hi, N - 1, i0))
    t = np.where(lo | hi, 0.0, t)
    i1 = np.minimum(i0 + 1, N - 1)
    return i0, i1, t


def _axis_weights_nodes(N: int, r: int):
    """Per fine node i (0..rN) of an axis: coarse nodes i0, i0 + 1 and the weight
    t of i0 + 1 (fine node at coarse coordinate i / r)."""
    i = np.arange(N * r + 1)
    i0 = np.minimum(i // r, N - 1)
    t = i / r - i0
    return i0, i0 + 1, t


def resample(grid_c, v, grid_f, kind: int) -> np.ndarray:
    """Carry a field from grid_c to grid_f = r * grid_c (integer r >= 1 per axis):
    the resolution change of the interpolation technique of Sec. 3 (a design
    optimised at low resolution becomes the start of the high-resolution run;
    Sec. 4.1 goes 128^3 -> 256^3 -> 512^3).  The paper does not state the
    interpolant; three are defined here:

    kind 0: element field, piecewise constant (each coarse element's value on its
            r^3 children; the mean is preserved exactly);
    kind 1: element field, trilinear between coarse cell centres, constant beyond
            the outermost centres (values stay in the range of the input);
    kind 2: nodal field, the coarse trilinear (Q1) function evaluated at the fine
            nodes (an exact embedding of the coarse finite-element space).
    Flat x-fastest arrays in the workloads' layout; FP64."""
    Nc = [int(g) for g in grid_c]
    Nf = [int(g) for g in grid_f]
    r = [f // c for f, c in zip(Nf, Nc)]
    if any(f != c * q or q < 1 for f, c, q in zip(Nf, Nc, r)):
        raise ValueError("grid_f must be an integer multiple of grid_c per axis")
    v = np.asarray(v, dtype=np.float64)
    if kind == 0:
        a = v.reshape(Nc[2], Nc[1], Nc[0])
        return np.repeat(np.repeat(np.repeat(a, r[2], axis=0), r[1], axis=1), r[0], axis=2).reshape(-1)
    if kind == 1:
        w = [_axis_weights_cells(Nc[k], r[k]) for k in range(3)]
        a = v.reshape(Nc[2], Nc[1], Nc[0])
    elif kind == 2:
        w = [_axis_weights_nodes(Nc[k], r[k]) for k in range(3)]
        a = v.reshape(Nc[2] + 1, Nc[1] + 1, Nc[0] + 1)
    else:
        raise ValueError("kind must be 0, 1 or 2")
    (x0, x1, tx), (y0, y1, ty), (z0, z1, tz) = w
    tx, ty, tz = tx[None, None, :], ty[None, :, None], tz[:, None, None]

    def at(zi, yi, xi):
        return a[np.ix_(zi, yi, xi)]

    # nested linear interpolation: x, then y, then z
    c00 = at(z0, y0, x0) * (1.0 - tx) + at(z0, y0, x1) * tx
    c10 = at(z0, y1, x0) * (1.0 - tx) + at(z0, y1, x1) * tx
    c01 = at(z1, y0, x0) * (1.0 - tx) + at(z1, y0, x1) * tx
    c11 = at(z1, y1, x0) * (1.0 - tx) + at(z1, y1, x1) * tx
    c0 = c00 * (1.0 - ty) + c10 * ty
    c1 = c01 * (1.0 - ty) + c11 * ty
    return (c0 * (1.0 - tz) + c1 * tz).reshape(-1)
