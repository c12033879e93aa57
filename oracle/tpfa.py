"""The paper's own discretisation (Sec. 2.2): cell-centred two-point flux
approximation (TPFA), the design-dependent heat source of Sec. 2.1 Eq. (1) and
the mean-temperature objective with its adjoint (Sec. 2.3, the LS1 / LS2
pair of Sec. 4).  Oracle (test infrastructure only), FP64, scipy sparse.

Unknowns: one temperature t_c per element (cell) c = i + Nx (j + Ny k), the
same index as the design x_c.

* Faces between cells a and b along axis d carry the flux
  v_F = -kappa_F (t_b - t_a) / h_d with the harmonic mean
  kappa_F = 2 / (1/kappa_a + 1/kappa_b) (Sec. 2.2 Eq. (4)); integrated over the
  face (area |F| = product of the other two edges) this gives the
  transmissibility tau_F = kappa_F |F| / h_d.
* Faces on Gamma_N carry no flux.  A face on Gamma_D carries the flux to the
  prescribed temperature over half a cell: tau = kappa_c |F| / (h_d / 2)
  (the reading of the velocity elimination at a Dirichlet face; DESIGN R25).
* Cell balance (Sec. 2.2 Eq. (5)): sum_F tau_F (t_c - t_nb) = f_c |K|, with the
  Dirichlet faces contributing tau (t_c - T_D): A t = q |K| + tau_D T_D.
* Source f_c = f0 (1 - x_c^p) (Sec. 2.1 Eq. (1)).
* Objective c = (1/M) sum_c t_c (Sec. 2.3 Eq. (6)); adjoint A u = 1/M (Eq. (7),
  A symmetric); sensitivity dc/dx_e = u^T (df/dx_e - dA/dx_e t + db_D/dx_e).

Which boundary faces are Dirichlet: a face on the box boundary whose centre
lies in the closed patch given by `dirichlet_faces` (the benchmark's centred
0.2 x 0.2 patch of z = 0, or a whole face).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem


def simp_source(x, p, f0):
    """Sec. 2.1 Eq. (1): f = f0 (1 - x^p) per cell."""
    x = np.asarray(x, dtype=np.float64)
    return f0 * (1.0 - x ** p)


def dirichlet_faces(grid, face: str = "z0", half_width: float = 0.1, centre=(0.5, 0.5)) -> dict:
    """Boolean masks of Dirichlet boundary faces, keyed by (axis, side): the
    cells whose face on that side of the box lies in Gamma_D.  'z0': the closed
    patch |x - cx| <= w, |y - cy| <= w of z = 0 (face centres, 1e-12 h
    tolerance); 'z0_full' / 'z1_full': a whole face; 'z0z1_full': both."""
    Nx, Ny, Nz = grid
    out = {}
    if face == "z0":
        xs = (np.arange(Nx) + 0.5) / Nx
        ys = (np.arange(Ny) + 0.5) / Ny
        tol = 1e-12 / max(Nx, Ny)
        inx = np.abs(xs - centre[0]) <= half_width + tol
        iny = np.abs(ys - centre[1]) <= half_width + tol
        m = np.zeros((Nz, Ny, Nx), dtype=bool)
        m[0][np.ix_(iny, inx)] = True
        out[(2, 0)] = m.reshape(-1)
    else:
        sides = {"z0_full": [0], "z1_full": [1], "z0z1_full": [0, 1]}[face]
        for s in sides:
            m = np.zeros((Nz, Ny, Nx), dtype=bool)
            m[0 if s == 0 else Nz - 1] = True
            out[(2, s)] = m.reshape(-1)
    return out


def _faces(grid):
    """Internal faces: (axis, cell a, cell b = a + stride) for every axis."""
    Nx, Ny, Nz = grid
    idx = np.arange(Nx * Ny * Nz).reshape(Nz, Ny, Nx)
    return [(0, idx[:, :, :-1].ravel(), idx[:, :, 1:].ravel()),
            (1, idx[:, :-1, :].ravel(), idx[:, 1:, :].ravel()),
            (2, idx[:-1, :, :].ravel(), idx[1:, :, :].ravel())]


def _area_over_h(h, d):
    hx, hy, hz = (float(v) for v in h)
    area = (hy * hz, hx * hz, hx * hy)[d]
    return area / (hx, hy, hz)[d]


def assemble(grid, h, kappa, dfaces):
    """The TPFA matrix A (M x M, SPD with a nonempty Dirichlet set) and the
    Dirichlet transmissibilities per face set {(axis, side): tau per cell}
    (the coefficients of T_D on the right-hand side)."""
    M = grid[0] * grid[1] * grid[2]
    kappa = np.asarray(kappa, dtype=np.float64)
    rows, cols, vals = [], [], []
    diag = np.zeros(M)
    for d, a, b in _faces(grid):
        tau = _area_over_h(h, d) * 2.0 / (1.0 / kappa[a] + 1.0 / kappa[b])
        rows += [a, b]
        cols += [b, a]
        vals += [-tau, -tau]
        np.add.at(diag, a, tau)
        np.add.at(diag, b, tau)
    tauD = {}
    for key, m in dfaces.items():
        tD = np.zeros(M)
        tD[m] = 2.0 * _area_over_h(h, key[0]) * kappa[m]
        tauD[key] = tD
        diag += tD
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(M, M))
    return (A + sp.diags(diag)).tocsr(), tauD


def _td(TD, key):
    """The prescribed temperature on the Dirichlet face set `key`: TD is a number
    (every set) or a dict {(axis, side): number or per-cell array}."""
    return TD[key] if isinstance(TD, dict) else TD


def build(grid, h, x, p, kmin, kmax, f0, dfaces, TD=0.0, source=None):
    """Problem bundle: kappa, A, the right-hand side b = f |K| + sum tau_D T_D.
    source (optional) replaces the design-dependent f0 (1 - x^p) per cell."""
    kappa = fem.simp_kappa(x, p, kmin, kmax)
    A, tauD = assemble(grid, h, kappa, dfaces)
    vol = float(h[0]) * float(h[1]) * float(h[2])
    f = simp_source(x, p, f0) if source is None else np.asarray(source, dtype=np.float64)
    b = f * vol
    for key, tD in tauD.items():
        b = b + tD * _td(TD, key)
    return dict(grid=tuple(grid), h=tuple(float(v) for v in h), x=np.asarray(x, float), p=float(p), kmin=float(kmin),
                kmax=float(kmax), f0=float(f0), TD=TD, kappa=kappa, A=A, tauD=tauD, b=b, dfaces=dfaces,
                source_given=source is not None)


def mean_temperature(t) -> float:
    """Sec. 2.3 Eq. (6): c = (1/M) sum_c t_c."""
    t = np.asarray(t, dtype=np.float64)
    return float(t.mean())


def adjoint_rhs(M: int) -> np.ndarray:
    """dc/dt = 1/M: the right-hand side of the adjoint system (LS2)."""
    return np.full(M, 1.0 / M)


def sensitivity(P, t, u) -> np.ndarray:
    """Sec. 2.3: dc/dx_e = u^T (df/dx_e - dA/dx_e t + db_D/dx_e) for every cell e,
    with t the state (A t = b) and u the adjoint (A u = 1/M).

    dkappa_e/dx_e = p x_e^(p-1) (kmax - kmin); for a face (e, nb) with
    tau = (|F|/h) 2 / (1/kappa_e + 1/kappa_nb), dtau/dkappa_e = tau^2 / (2 (|F|/h) kappa_e^2),
    contributing -dtau (u_e - u_nb)(t_e - t_nb); a Dirichlet face of e with
    tau_D = 2 (|F|/h) kappa_e contributes -dtau_D u_e (t_e - T_D); the source
    contributes -f0 p x_e^(p-1) |K| u_e."""
    grid, h = P["grid"], P["h"]
    x, p = P["x"], P["p"]
    kappa = P["kappa"]
    t = np.asarray(t, float)
    u = np.asarray(u, float)
    M = x.size
    xp1 = x ** (p - 1.0)
    dk = p * xp1 * (P["kmax"] - P["kmin"])
    g = np.zeros(M)
    for d, a, b in _faces(grid):
        ah = _area_over_h(h, d)
        tau = ah * 2.0 / (1.0 / kappa[a] + 1.0 / kappa[b])
        w = (u[a] - u[b]) * (t[a] - t[b])
        np.add.at(g, a, -tau ** 2 / (2.0 * ah * kappa[a] ** 2) * w)
        np.add.at(g, b, -tau ** 2 / (2.0 * ah * kappa[b] ** 2) * w)
    for key, m in P["dfaces"].items():
        ah = _area_over_h(h, key[0])
        td = np.broadcast_to(np.asarray(_td(P["TD"], key), dtype=np.float64), (M,))
        g[m] += -2.0 * ah * u[m] * (t[m] - td[m])
    vol = float(h[0]) * float(h[1]) * float(h[2])
    src = 0.0 if P["source_given"] else P["f0"] * p * xp1 * vol * u
    return dk * g - src


def mmg_problem(P, b: int = 4) -> dict:
    """The TPFA system as a problem for oracle.mmg.MMG (the algebraic
    construction of Sec. 3 on the paper's own discretisation): unknowns are the
    cells, level-1 blocks are b^3 cells (the block grid must divide), the mass of
    Eq. (8) is the kappa-weighted cell volume kappa_c |K| (the cell-centred
    counterpart of the lumped nodal mass), no unknown is eliminated (Dirichlet
    data enter through the faces), and the internal Neumann form of a block is
    its diagonal block of A minus the row sums -- exactly the flux over the
    block's internal faces, as Eq. (8) states for TPFA."""
    Nx, Ny, Nz = P["grid"]
    if Nx % b or Ny % b or Nz % b:
        raise ValueError("the grid must be a multiple of the block size")
    c = np.arange(Nx * Ny * Nz)
    i, j, k = c % Nx, (c // Nx) % Ny, c // (Nx * Ny)
    sx, sy, sz = Nx // b, Ny // b, Nz // b
    blk = (i // b) + sx * ((j // b) + sy * (k // b))
    vol = P["h"][0] * P["h"][1] * P["h"][2]
    return dict(grid=P["grid"], h=P["h"], A=P["A"], b=P["b"], mask=np.zeros(c.size, dtype=bool),
                mass=P["kappa"] * vol, blocks=(blk, (sx, sy, sz)))
