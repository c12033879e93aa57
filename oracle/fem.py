"""Q1 (trilinear) finite elements for -div(kappa grad T) = q on a box grid.

Oracle (test infrastructure only).  Everything here is assembled element by
element from the textbook definition A = sum_e kappa_e K0_e, in FP64, with
scipy sparse matrices.

Paper anchors
  * SIMP conductivity, Sec. 2.1 Eq. (1):  kappa = kL + x^p (kH - kL).
  * Linear system A t = f, Sec. 2.2 Eq. (5).  The paper discretises with TPFA
    finite volumes; this oracle uses trilinear nodal elements on the same
    structured grid (one unknown per grid node), which keeps the system SPD
    with the same SIMP law and the same Dirichlet/Neumann boundary data.
  * Objective and adjoint, Sec. 2.3 Eqs. (6)-(7): for the compliance
    c = f^T u with a design-independent load the adjoint equals the state and
    dc/dx_e = -p x_e^(p-1) (kH - kL) u_e^T K0 u_e.

Index conventions: node n = i + nx*(j + ny*k) with nx = Nx+1 (x fastest),
element e = ex + Nx*(ey + Ny*ez), local node a = ax + 2*ay + 4*az of element
(ex,ey,ez) is global node (ex+ax, ey+ay, ez+az).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])            # 1-D stiffness * h
_M1 = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])  # 1-D mass / h


def element_matrix(h) -> np.ndarray:
    """8x8 Q1 stiffness of one box element of size hx*hy*hz, unit conductivity.

    K0 = (hy hz/hx) m(x)m(x)k + (hx hz/hy) m(x)k(x)m + (hx hy/hz) k(x)m(x)m
    (Kronecker products ordered z, y, x so that the row index is ax+2ay+4az),
    with the exact 1-D stiffness k/h and mass h*m of linear elements.
    Pinned against 2x2x2 Gauss quadrature of grad(phi_a).grad(phi_b) and the
    closed-form cube entries/eigenvalues in tests.
    """
    hx, hy, hz = (float(v) for v in h)
    K = (hy * hz / hx) * np.kron(_M1, np.kron(_M1, _K1))
    K += (hx * hz / hy) * np.kron(_M1, np.kron(_K1, _M1))
    K += (hx * hy / hz) * np.kron(_K1, np.kron(_M1, _M1))
    return K


def simp_kappa(x, p, kmin, kmax) -> np.ndarray:
    """Sec. 2.1 Eq. (1): kappa_e = kmin + x_e^p (kmax - kmin)."""
    x = np.asarray(x, dtype=np.float64)
    return kmin + x ** p * (kmax - kmin)


def element_nodes(grid) -> np.ndarray:
    """(M, 8) global node ids of every element, local order ax+2ay+4az."""
    Nx, Ny, Nz = grid
    nx, ny = Nx + 1, Ny + 1
    ez, ey, ex = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx),
                             indexing="ij")
    base = (ex + nx * (ey + ny * ez)).reshape(-1)
    out = np.empty((base.size, 8), dtype=np.int64)
    for a in range(8):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        out[:, a] = base + ax + nx * (ay + ny * az)
    return out


def n_nodes(grid) -> int:
    return (grid[0] + 1) * (grid[1] + 1) * (grid[2] + 1)


def assemble_neumann(grid, h, kappa) -> sp.csr_matrix:
    """A_N = sum_e kappa_e K0 scattered on the element's 8 nodes (no BCs).

    This is the all-Neumann (singular) operator; its rows sum to zero.
    """
    K0 = element_matrix(h)
    en = element_nodes(grid)
    M = en.shape[0]
    rows = np.repeat(en, 8, axis=1).reshape(-1)
    cols = np.tile(en, (1, 8)).reshape(-1)
    vals = (np.asarray(kappa, dtype=np.float64)[:, None] * K0.reshape(1, 64)).reshape(-1)
    n = n_nodes(grid)
    A = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def load_vector(grid, h, source) -> np.ndarray:
    """f_i = int q phi_i = sum_{e contains i} q_e hx hy hz / 8 (exact for
    element-wise constant q, since each trilinear shape integrates to vol/8)."""
    vol = float(h[0]) * float(h[1]) * float(h[2])
    en = element_nodes(grid)
    f = np.zeros(n_nodes(grid))
    np.add.at(f, en.reshape(-1), np.repeat(np.asarray(source, float) * vol / 8.0, 8))
    return f


def lumped_kappa_mass(grid, h, kappa) -> np.ndarray:
    """m_i = sum_{e contains i} kappa_e hx hy hz / 8: the diagonal (lumped)
    kappa-weighted mass that discretises int kappa Phi q dV in Sec. 3 Eq. (8)."""
    return load_vector(grid, h, kappa)


def dirichlet_system(A_neu, f, mask, values=None):
    """Eliminate Dirichlet nodes: rows/columns of D are replaced by identity,
    b_F = f_F - A_FD T_D, b_D = T_D (Sec. 2.1 boundary data on Gamma_D).

    Returns (A, b) with A = P_F A_N P_F + P_D.
    """
    mask = np.asarray(mask).astype(bool)
    n = A_neu.shape[0]
    TD = np.zeros(n) if values is None else np.where(mask, values, 0.0)
    free = (~mask).astype(np.float64)
    PF = sp.diags(free)
    A = (PF @ A_neu @ PF + sp.diags(mask.astype(np.float64))).tocsr()
    b = free * (f - A_neu @ TD) + mask * TD
    return A, b


def build_problem(grid, h, x, p, kmin, kmax, mask, source, values=None):
    """Convenience bundle: kappa, A_N, A (Dirichlet-eliminated), f, b, mass."""
    kappa = simp_kappa(x, p, kmin, kmax)
    A_neu = assemble_neumann(grid, h, kappa)
    f = load_vector(grid, h, source)
    A, b = dirichlet_system(A_neu, f, mask, values)
    return dict(grid=tuple(grid), h=tuple(float(v) for v in h), x=np.asarray(x, float),
                p=float(p), kmin=float(kmin), kmax=float(kmax),
                kappa=kappa, A_neu=A_neu, A=A, f=f, b=b,
                mask=np.asarray(mask).astype(bool),
                mass=lumped_kappa_mass(grid, h, kappa))


def operator_rows(grid, h, kappa, mask, u, rows, absolute=False, chunk=1 << 21) -> np.ndarray:
    """(A u)_i on the listed nodes i for the Dirichlet-eliminated operator
    A = P_F A_N P_F + P_D of Sec. 2.2 Eq. (5) with the Gamma_D data of Sec. 2.1,
    evaluated row by row from the element matrices, without assembling A: a
    free row sums kappa_e K0[a, b] u_b over the (up to) eight elements e that
    contain node i (as their local node a) and over their free nodes b; a
    Dirichlet row returns u_i.  absolute=True evaluates (|A| |u|)_i, the scale
    of a row's rounding error.  Serves spot checks of outputs too large for
    the assembled matrix.
    """
    Nx, Ny, Nz = grid
    nx, ny = Nx + 1, Ny + 1
    K0 = element_matrix(h)
    if absolute:
        K0 = np.abs(K0)
    kappa = np.asarray(kappa, dtype=np.float64)
    mask = np.asarray(mask).astype(bool)
    u = np.asarray(u, dtype=np.float64)
    if absolute:
        u = np.abs(u)
    rows = np.asarray(rows, dtype=np.int64).reshape(-1)
    out = np.empty(rows.size)
    for c0 in range(0, rows.size, chunk):
        r = rows[c0:c0 + chunk]
        ix, iy, iz = r % nx, (r // nx) % ny, r // (nx * ny)
        y = np.zeros(r.size)
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            ex, ey, ez = ix - ax, iy - ay, iz - az
            ok = (ex >= 0) & (ey >= 0) & (ez >= 0) & (ex < Nx) & (ey < Ny) & (ez < Nz)
            ke = np.where(ok, kappa[np.where(ok, ex + Nx * (ey + Ny * ez), 0)], 0.0)
            for b in range(8):
                bx, by, bz = b & 1, (b >> 1) & 1, (b >> 2) & 1
                nb = np.where(ok, (ex + bx) + nx * ((ey + by) + ny * (ez + bz)), 0)
                ub = np.where(mask[nb], 0.0, u[nb])
                y += ke * (K0[a, b] * ub)
        out[c0:c0 + r.size] = np.where(mask[r], u[r], y)
    return out


def load_rows(grid, h, source, rows) -> np.ndarray:
    """f_i of load_vector on the listed nodes only, summed over the (up to) eight
    elements that contain node i; for spot checks of grids too large for f."""
    Nx, Ny, Nz = grid
    nx, ny = Nx + 1, Ny + 1
    vol = float(h[0]) * float(h[1]) * float(h[2])
    src = np.asarray(source, dtype=np.float64)
    r = np.asarray(rows, dtype=np.int64).reshape(-1)
    ix, iy, iz = r % nx, (r // nx) % ny, r // (nx * ny)
    out = np.zeros(r.size)
    for a in range(8):
        ex, ey, ez = ix - (a & 1), iy - ((a >> 1) & 1), iz - (a >> 2)
        ok = (ex >= 0) & (ey >= 0) & (ez >= 0) & (ex < Nx) & (ey < Ny) & (ez < Nz)
        e = np.where(ok, ex + Nx * (ey + Ny * ez), 0)
        out += np.where(ok, src[e] * vol / 8.0, 0.0) if src.ndim else np.where(ok, float(src) * vol / 8.0, 0.0)
    return out


def sensitivity_at(grid, h, x_e, p, kmin, kmax, u, elems) -> np.ndarray:
    """sensitivity() on the listed elements only: x_e are those elements'
    densities, u the whole nodal solution; for spot checks of large grids."""
    Nx, Ny, _ = grid
    nx, ny = Nx + 1, Ny + 1
    K0 = element_matrix(h)
    e = np.asarray(elems, dtype=np.int64).reshape(-1)
    ex, ey, ez = e % Nx, (e // Nx) % Ny, e // (Nx * Ny)
    base = ex + nx * (ey + ny * ez)
    ue = np.empty((e.size, 8))
    for a in range(8):
        ue[:, a] = np.asarray(u, float)[base + (a & 1) + nx * (((a >> 1) & 1) + ny * (a >> 2))]
    E = np.einsum("ea,ab,eb->e", ue, K0, ue)
    x = np.asarray(x_e, float)
    return -p * x ** (p - 1.0) * (kmax - kmin) * E


def compliance(f, u) -> float:
    """c = f^T u; for q = 1 on the unit cube this equals int u_h dV, the mean
    temperature of Sec. 2.3 Eq. (6) (sum_i phi_i = 1)."""
    return float(np.dot(f, u))


def element_energy(grid, h, u) -> np.ndarray:
    """u_e^T K0 u_e for every element (unit conductivity)."""
    K0 = element_matrix(h)
    ue = np.asarray(u, float)[element_nodes(grid)]
    return np.einsum("ea,ab,eb->e", ue, K0, ue)


def sensitivity(grid, h, x, p, kmin, kmax, u) -> np.ndarray:
    """Sec. 2.3 adjoint formula u^T(df/dx - dA/dx t) with df/dx = 0 and adjoint
    = state (compliance, homogeneous Dirichlet data):
        dc/dx_e = -p x_e^(p-1) (kmax - kmin) u_e^T K0 u_e.
    Pinned by central finite differences and the Euler identity in tests."""
    x = np.asarray(x, float)
    return -p * x ** (p - 1.0) * (kmax - kmin) * element_energy(grid, h, u)
