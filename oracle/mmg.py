"""Multiscale multigrid (MMG) preconditioner, plain FP64 (oracle, test only).

Follows Sec. 3 of the paper step by step:

* Grid hierarchy (Sec. 3, nested grids K^(0) ⊃ K^(1) ⊃ ...): level 1 cells are
  blocks of b^3 fine elements; level l >= 2 cells are groups of g^3 level-(l-1)
  cells.  Fine *nodes* are partitioned among level-1 blocks by
  block(i) = min(i // b, N/b - 1) per axis (the last block of an axis also
  takes the closing node plane); Dirichlet nodes belong to no block.
* Coarse spectral problem, Eq. (8): on each block B, the Neumann form over the
  faces/couplings internal to B against the kappa-weighted diagonal mass.
  Algebraically: Ã_B = A_BB - diag(A_BB 1) (couplings leaving B and to
  Dirichlet nodes removed, so constants are in the null space) and
  M_B = diag(m_i), m_i = sum_{e ∋ i} kappa_e |e| / 8.  The L_1 eigenvectors of
  smallest eigenvalue, normalised to Phi^T M Phi = I, are the rows of R_c.
* Coarse-coarse spectral problem, Eq. (9): on each group G, the same Neumann
  form (internal to G) restricted to the span of the previous level's basis
  functions supported in G.  With the M-normalised basis the right-hand side
  is the identity (the "mass trick" after Eq. (9)), so it is a standard
  symmetric eigenproblem.  Rows of R_cc R_c are the composite eigenfunctions.
  Levels beyond the paper's three grids repeat this construction.
* Galerkin coarse operators A_c = R_c A R_c^T, A_cc = R_cc A_c R_cc^T (Sec. 3).
* Smoothed V-cycle, Algorithm 1 (generalised to any number of levels, with
  the coarsest "correction" read as a solve with A_cc, i.e. A_cc^{-1} r_cc).
  Coarse levels: nu_coarse sweeps on level 1, doubled per level below it, and
  two coarse corrections per visit from level 3 on (a W-cycle: the deep levels
  stand in for the paper's direct coarse-coarse solve, so they are solved more
  accurately than one V-cycle would).
  Fine smoother: nu damped-Jacobi sweeps, or (default) Chebyshev-accelerated
  Jacobi of degree m on [lmax/30, 1.1 lmax] of D^-1 A -- the paper smooths
  with block-Jacobi inside PETSc's Krylov smoothers (Sec. 4), whose
  multigrid default is Chebyshev; coarse smoother: l1-block-Jacobi over each
  cell's L x L block.  Both are polynomials in / inverses of symmetric
  operators applied identically before and after, so S^{-T} = S^{-1}.  Coarsest: dense Cholesky (the paper uses a
  sparse LU; A_cc is SPD so the solves agree).

Parity pins (tests/test_oracle_mmg.py): two-level exactness with a complete
local basis, M-orthonormality, eigen-residuals, zero row sums / SPSD of the
local Neumann matrices, V-cycle symmetry and positivity, agreement of the
algorithmic V-cycle with its closed product form on small grids, and the
Galerkin-orthogonality invariant of the coarse initial guess.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

import workloads as W
import scipy.linalg as sla
import scipy.sparse as sp


@dataclass
class MMGOptions:
    block: int = 4                      # b: block edge in fine elements
    nvec: tuple = (4, 17)               # L_1, L_2, ... (one per coarse level)
    group: tuple = (2,)                 # g_2, g_3, ... (one per level >= 2)
    nu_fine: int = 2                    # damped-Jacobi sweeps (smoother = "jacobi")
    nu_coarse: int = 1
    nu_growth: int = 2                  # coarse sweeps on level l: nu_coarse * nu_growth^(l-1), at most 64
    w_from: int = 3                     # levels >= w_from make two coarse corrections (0: V-cycle)
    omega: float = 2.0 / 3.0
    smoother: str = "jacobi"            # fine smoother: "jacobi" or "chebyshev"
    cheb_degree: int = 5                # Chebyshev: matrix-vector products per smoothing
    cheb_ratio: float = 30.0            # interval [lmax / ratio, 1.1 lmax] of D^-1 A
    power_iters: int = 15               # power iterations for lmax(D^-1 A)
    eig_threshold: float = 0.0          # > 0: adaptive basis count (see kept_count); 0: L_l per cell

    def __post_init__(self):
        self.nvec = tuple(int(v) for v in self.nvec)
        self.group = tuple(int(v) for v in self.group)
        if len(self.group) != len(self.nvec) - 1:
            raise ValueError("need one group size per level >= 2")


def default_options(N: int, smoother: str = "chebyshev") -> MMGOptions:
    """Hierarchy used for an N^3 grid: b = 4, L_1 = 4, then groups of 2^3
    cells down to a coarsest level of 4^3 cells (8^3 cells when there are more
    than 32^3 blocks) with L = 17 (1,088 or 8,704 unknowns); the second level
    keeps L = 8 when the hierarchy has more than three grids and L = 17 from
    the third level on."""
    nb = N // 4
    levels = []
    m = nb
    stop = 8 if nb > 32 else 4
    while m > stop:
        m //= 2
        levels.append(m)
    if not levels:
        return MMGOptions(block=4, nvec=(4,), group=(), smoother=smoother)
    nvec = [4]
    for i, _ in enumerate(levels):
        nvec.append(8 if (i == 0 and len(levels) > 1) else 17)
    return MMGOptions(block=4, nvec=tuple(nvec), group=(2,) * len(levels), smoother=smoother)


@dataclass
class Level:
    shape: tuple                      # cells per axis at this level
    L: int                            # vectors per cell
    P: sp.csr_matrix = None           # prolongation from this level to the previous one
    A: sp.csr_matrix = None           # Galerkin operator at this level
    active: np.ndarray = None         # per-dof flag (False: zero basis vector)
    smoother: list = field(default_factory=list)  # per-cell inverse of the l1 block
    eigvals: list = field(default_factory=list)


POWER_SEED = 101


def power_start(n):
    """Seeded start vector of the power iteration: u_i - 1/2 with u the SplitMix64
    uniforms of stream POWER_SEED at the natural node index (the shared input
    generator).  A random start has weight on the top of the spectrum of D^-1 A;
    a smooth or periodic one does not on uniform media, where 15 iterations then
    underestimate lmax by 12-17% and the Chebyshev smoother amplifies the top modes."""
    return W.uniform01(POWER_SEED, n) - 0.5


def lmax_estimate(A, D, free, iters):
    """Power iteration for the largest eigenvalue of D^-1 A on the free nodes:
    v <- D^-1 A v / ||D^-1 A v||, estimate ||D^-1 A v|| for the last unit v."""
    v = power_start(A.shape[0]) * free
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(iters):
        w = (A @ v) / D * free
        lam = np.linalg.norm(w)
        v = w / lam
    return lam


def chebyshev_coefficients(lmax, ratio, degree):
    """Chebyshev smoother on [lmax/ratio, 1.1 lmax] for D^-1 A, as the
    three-term recurrence  e_{k+1} = e_k + a_k (e_k - e_{k-1}) + b_k D^-1 (r - A e_k)
    (a_0 = 0).  Its error propagation is the scaled Chebyshev polynomial
    T_m((hi + lo - 2 lam)/(hi - lo)) / T_m((hi + lo)/(hi - lo)), m = degree.
    Returns lists (a, b) of length degree."""
    lo, hi = lmax / ratio, 1.1 * lmax
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    a, b = [0.0], [1.0 / theta]
    for _ in range(1, degree):
        rho_new = 1.0 / (2.0 * sigma - rho)
        a.append(rho_new * rho)
        b.append(2.0 * rho_new / delta)
        rho = rho_new
    return a, b


def node_blocks(grid, b, mask):
    """Level-1 cell (block) id of every fine node, -1 for Dirichlet nodes."""
    Nx, Ny, Nz = grid
    if Nx % b or Ny % b or Nz % b:
        raise ValueError("grid must be a multiple of the block size")
    nbx, nby, nbz = Nx // b, Ny // b, Nz // b
    bx = np.minimum(np.arange(Nx + 1) // b, nbx - 1)
    by = np.minimum(np.arange(Ny + 1) // b, nby - 1)
    bz = np.minimum(np.arange(Nz + 1) // b, nbz - 1)
    BZ, BY, BX = np.meshgrid(bz, by, bx, indexing="ij")
    blk = (BX + nbx * (BY + nby * BZ)).reshape(-1)
    blk = np.where(np.asarray(mask).astype(bool), -1, blk)
    return blk, (nbx, nby, nbz)


def _sign_fix(v):
    """Make the entry of largest magnitude (lowest index on ties) positive."""
    k = int(np.argmax(np.abs(v)))
    return -v if v[k] < 0 else v


def _mgs(V, W=None):
    """Modified Gram-Schmidt of the columns of V in the inner product
    <a,b> = a^T diag(W) b (Euclidean if W is None), FP64."""
    V = V.copy()
    w = np.ones(V.shape[0]) if W is None else W
    for j in range(V.shape[1]):
        for i in range(j):
            V[:, j] -= (V[:, i] * w) @ V[:, j] * V[:, i]
        nrm = np.sqrt((V[:, j] * w) @ V[:, j])
        V[:, j] /= nrm
    return V


def _blocks(prob, opts: MMGOptions):
    """Level-1 cells of the unknowns: the Q1 node blocks (R4), or the partition a
    problem supplies as prob["blocks"] = (block id per unknown, -1 for none;
    block grid shape) -- e.g. blocks of b^3 cells for the cell-centred TPFA
    unknowns (oracle.tpfa.mmg_problem).  Everything after the partition is
    algebraic: the Neumann form of each block, the mass, the groups."""
    if "blocks" in prob:
        return prob["blocks"]
    return node_blocks(prob["grid"], opts.block, prob["mask"])


def cell_size(prob, opts: MMGOptions, level: int) -> float:
    """Edge H_l of a level-l cell: b max(h) on level 1, times g_2 ... g_l below."""
    H = opts.block * max(prob["h"])
    for g in opts.group[:level - 1]:
        H *= g
    return H


def kept_count(w, L: int, thr: float) -> int:
    """Adaptive local basis (the GMsFEM-style alternative to a fixed L): of the
    ascending local eigenvalues w, keep those with w H^2 <= tau (thr = tau / H^2),
    at most L (the cell's capacity) and at least one; thr <= 0 keeps
    min(L, len(w)).  In a high-contrast cell the eigenvalues of the
    kappa-weighted Neumann problem split into one near zero per high-conductivity
    component (kappa_min / kappa_max times the cell scale) and the rest above
    about pi^2 / H^2 (in the kappa-mass norm the constant is a combination of
    the components' indicators), so a threshold between the two keeps one
    vector per component."""
    k = min(L, len(w))
    if thr <= 0.0 or k == 0:
        return k
    c = 0
    while c < k and w[c] <= thr:
        c += 1
    return max(c, 1)


def level1_basis(prob, opts: MMGOptions):
    """Eq. (8) on every block: returns (P1 (n0 x n1), active, eigvals, blk)."""
    A = prob["A"].tocsr()
    mass = prob["mass"]
    blk, shape = _blocks(prob, opts)
    nblk = shape[0] * shape[1] * shape[2]
    L = opts.nvec[0]
    order = np.argsort(blk, kind="stable")
    counts = np.bincount(blk[blk >= 0], minlength=nblk)
    starts = np.concatenate([[0], np.cumsum(counts)])
    first_free = int(np.sum(blk < 0))
    rows, cols, vals = [], [], []
    active = np.zeros(nblk * L, dtype=bool)
    eigs = []
    for c in range(nblk):
        idx = order[first_free + starts[c]: first_free + starts[c + 1]]
        n = idx.size
        if n == 0:
            eigs.append(np.zeros(0))
            continue
        ABB = A[idx][:, idx].toarray()
        At = ABB - np.diag(ABB.sum(axis=1))          # internal Neumann form
        m = mass[idx]
        s = 1.0 / np.sqrt(m)
        C = At * s[:, None] * s[None, :]
        w, V = np.linalg.eigh(C)
        k = kept_count(w, L, opts.eig_threshold / cell_size(prob, opts, 1) ** 2)
        Phi = V[:, :k] * s[:, None]
        Phi = _mgs(Phi, m)                           # Phi^T M Phi = I
        for j in range(k):
            phi = _sign_fix(Phi[:, j])
            rows.append(idx)
            cols.append(np.full(n, c * L + j))
            vals.append(phi)
            active[c * L + j] = True
        eigs.append(w[:k])
    n0 = A.shape[0]
    P1 = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                       shape=(n0, nblk * L))
    return P1, active, eigs, blk, shape


def _galerkin(A, P, active):
    Ac = (P.T @ A @ P).tocsr()
    Ac = Ac.tolil()
    for d in np.flatnonzero(~active):
        Ac[d, d] = 1.0
    return Ac.tocsr()


def coarse_level_basis(prob, Pcomp, fine_cell, prev_shape, prev_L, prev_active,
                       g, L, thr=0.0):
    """Eq. (9) on every group of g^3 previous-level cells.

    fine_cell: previous-level cell id of each fine node (-1 for Dirichlet).
    Pcomp: composite prolongation fine <- previous level (n0 x n_prev).
    thr: the adaptive basis threshold tau / H^2 of this level (kept_count).
    Returns (Psi (n_prev x n_new), active_new, eigvals, new fine_cell, shape).
    """
    A = prob["A"].tocsr()
    mx, my, mz = prev_shape
    if mx % g or my % g or mz % g:
        raise ValueError("cell counts must be multiples of the group size")
    sx, sy, sz = mx // g, my // g, mz // g
    ngrp = sx * sy * sz
    cx = np.arange(mx * my * mz) % mx
    cy = (np.arange(mx * my * mz) // mx) % my
    cz = np.arange(mx * my * mz) // (mx * my)
    cell_group = (cx // g) + sx * ((cy // g) + sy * (cz // g))
    fine_group = np.where(fine_cell >= 0, cell_group[np.maximum(fine_cell, 0)], -1)
    Pc = Pcomp.tocsc()
    rows, cols, vals = [], [], []
    active = np.zeros(ngrp * L, dtype=bool)
    eigs = []
    # members of every group in increasing index order (a stable sort by group id
    # lists the same indices as a scan for each id, in one pass)
    cell_order = np.argsort(cell_group, kind="stable")
    cell_start = np.concatenate([[0], np.cumsum(np.bincount(cell_group, minlength=ngrp))])
    fine_order = np.argsort(fine_group, kind="stable")
    n_dir = int(np.sum(fine_group < 0))
    fine_start = n_dir + np.concatenate([[0], np.cumsum(np.bincount(fine_group[fine_group >= 0],
                                                                     minlength=ngrp))])
    for G in range(ngrp):
        cells = cell_order[cell_start[G]:cell_start[G + 1]]
        # local order: lx + g*ly + g^2*lz  (cells are already x-fastest sorted)
        key = (cx[cells] % g) + g * ((cy[cells] % g) + g * (cz[cells] % g))
        cells = cells[np.argsort(key)]
        dofs = (cells[:, None] * prev_L + np.arange(prev_L)[None, :]).reshape(-1)
        act = prev_active[dofs]
        fine = fine_order[fine_start[G]:fine_start[G + 1]]
        PG = Pc[:, dofs].tocsr()[fine].toarray()     # composite basis on G
        AGG = A[fine][:, fine]
        NG = AGG - sp.diags(np.asarray(AGG.sum(axis=1)).ravel())  # Neumann form internal to G
        At = PG.T @ (NG @ PG)
        ia = np.flatnonzero(act)
        Ata = At[np.ix_(ia, ia)]
        Ata = 0.5 * (Ata + Ata.T)
        w, V = np.linalg.eigh(Ata)
        k = kept_count(w, L, thr)
        Vk = _mgs(V[:, :k])
        for j in range(k):
            v = _sign_fix(Vk[:, j])
            rows.append(dofs[ia])
            cols.append(np.full(ia.size, G * L + j))
            vals.append(v)
            active[G * L + j] = True
        eigs.append(w[:k])
    n_prev = mx * my * mz * prev_L
    Psi = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(n_prev, ngrp * L))
    return Psi, active, eigs, fine_group, (sx, sy, sz)


def l1_block_inverses(A, shape, L):
    """Per cell: inverse of (A_cc + diag(sum over off-cell |a_ij|)) (FP64)."""
    A = A.tocsr()
    ncell = shape[0] * shape[1] * shape[2]
    out = []
    Aabs = abs(A)
    rowabs = np.asarray(Aabs.sum(axis=1)).ravel()
    for c in range(ncell):
        d = np.arange(c * L, (c + 1) * L)
        D = A[d][:, d].toarray()
        inside = np.asarray(Aabs[d][:, d].sum(axis=1)).ravel()
        D = D + np.diag(rowabs[d] - inside)
        out.append(np.linalg.inv(D))
    return out


def _given_level(P, shape, L):
    """A level whose basis is given (not computed from Eq. (8) / Eq. (9)):
    a dof is active when its basis column is nonzero."""
    P = sp.csr_matrix(P)
    act = np.asarray(abs(P).sum(axis=0)).ravel() > 0
    return P, act, [], shape


class MMG:
    """The full hierarchy for one problem; ``apply(r)`` is one V-cycle.

    ``bases`` (optional): prolongations to use instead of the local spectral
    bases -- ``bases[0]`` the level-1 Phi (n0 x n1, columns cell * L_1 + j),
    ``bases[l]`` the Psi of level l + 1 (n_l x n_{l+1}, columns group * L + j)
    -- for the same cells and vector counts as the options.  Everything that
    follows the bases (Galerkin operators, smoothers, the cycle of Algorithm 1,
    the coarse guess) is computed as usual.  This lets a test evaluate the
    cycle's arithmetic on another implementation's bases."""

    def __init__(self, prob, opts: MMGOptions | None = None, bases=None):
        N = prob["grid"][0]
        self.opts = opts or default_options(N)
        self.prob = prob
        A = prob["A"].tocsr()
        self.A0 = A
        self.D0 = A.diagonal().copy()
        o = self.opts
        if bases is None:
            P1, act, eig, fine_cell, shape = level1_basis(prob, o)
        else:
            _, shape = _blocks(prob, o)
            P1, act, eig, shape = _given_level(bases[0], shape, o.nvec[0])
            fine_cell = None
        if o.smoother == "chebyshev":
            free = (~prob["mask"]).astype(float)
            self.lmax = lmax_estimate(A, self.D0, free, o.power_iters)
            self.cheb = chebyshev_coefficients(self.lmax, o.cheb_ratio, o.cheb_degree)
        self.levels = [Level(shape=shape, L=o.nvec[0], P=P1, active=act, eigvals=eig)]
        self.levels[0].A = _galerkin(A, P1, act)
        Pcomp = P1
        for li, (g, L) in enumerate(zip(o.group, o.nvec[1:])):
            prev = self.levels[-1]
            if bases is None:
                thr = o.eig_threshold / cell_size(prob, o, li + 2) ** 2
                Psi, act, eig, fine_cell, shape = coarse_level_basis(
                    prob, Pcomp, fine_cell, prev.shape, prev.L, prev.active, g, L, thr)
            else:
                shape = tuple(m // g for m in prev.shape)
                Psi, act, eig, shape = _given_level(bases[li + 1], shape, L)
            lev = Level(shape=shape, L=L, P=Psi, active=act, eigvals=eig)
            lev.A = _galerkin(prev.A, Psi, act)
            self.levels.append(lev)
            Pcomp = (Pcomp @ Psi).tocsr()
        self.Pcomp = Pcomp
        for lev in self.levels[:-1]:
            lev.smoother = l1_block_inverses(lev.A, lev.shape, lev.L)
        Ac = self.levels[-1].A.toarray()
        self.coarse_chol = sla.cho_factor(Ac, lower=True)

    # -- pieces of Algorithm 1 -------------------------------------------------
    def coarse_solve(self, r):
        return sla.cho_solve(self.coarse_chol, r)

    def _smooth(self, l, r, e):
        """One sweep e <- e + S^{-1}(r - A_l e) on grid l (0 = fine)."""
        if l == 0:
            return e + self.opts.omega * (r - self.A0 @ e) / self.D0
        lev = self.levels[l - 1]
        res = r - lev.A @ e
        out = e.copy()
        L = lev.L
        for c, Dinv in enumerate(lev.smoother):
            s = slice(c * L, (c + 1) * L)
            out[s] += Dinv @ res[s]
        return out

    def _A(self, l):
        return self.A0 if l == 0 else self.levels[l - 1].A

    def _chebyshev(self, r, e):
        """Chebyshev smoothing on the fine grid from the iterate e."""
        a, b = self.cheb
        prev = e
        for k in range(len(a)):
            new = e + b[k] * (r - self.A0 @ e) / self.D0
            if k > 0:
                new = new + a[k] * (e - prev)
            prev, e = e, new
        return e

    def _presmooth(self, l, r):
        e = np.zeros_like(r)
        if l == 0 and self.opts.smoother == "chebyshev":
            return self._chebyshev(r, e)
        for _ in range(self._sweeps(l)):
            e = self._smooth(l, r, e)
        return e

    def _postsmooth(self, l, r, e):
        if l == 0 and self.opts.smoother == "chebyshev":
            return self._chebyshev(r, e)
        for _ in range(self._sweeps(l)):
            e = self._smooth(l, r, e)
        return e

    def _sweeps(self, l):
        """Smoothing sweeps on level l: nu_fine on the fine grid; nu_coarse on level 1,
        multiplied by nu_growth per level below it (at most 64)."""
        if l == 0:
            return self.opts.nu_fine
        return min(64, self.opts.nu_coarse * self.opts.nu_growth ** (l - 1))

    def vcycle(self, r, l=0):
        """Algorithm 1 on grids l, l+1, ..., coarsest (recursive)."""
        nlev = len(self.levels)
        if l == nlev:
            return self.coarse_solve(r)
        A = self._A(l)
        e = self._presmooth(l, r)                 # pre-smoothing (from e = 0)
        P = self.levels[l].P
        # one coarse correction (V-cycle); two on coarse levels >= w_from (W-cycle) unless
        # the next level is the direct solve, where a second Galerkin correction is zero
        w = self.opts.w_from
        reps = 2 if (l >= 1 and w > 0 and l >= w and l + 1 < nlev) else 1
        for _ in range(reps):
            rc = P.T @ (r - A @ e)                # restriction of the residual
            ec = self.vcycle(rc, l + 1)
            e = e + P @ ec                        # prolongation
        e = self._postsmooth(l, r, e)             # post-smoothing (S^{-T} = S^{-1})
        return e

    __call__ = vcycle

    def coarse_guess(self, b, u_prev=None):
        """u0 = P A_L^{-1} P^T b (or the same correction of u_prev): the
        Galerkin coarsest-level solution interpolated to the fine grid."""
        P = self.Pcomp
        if u_prev is None:
            return P @ self.coarse_solve(P.T @ b)
        return u_prev + P @ self.coarse_solve(P.T @ (b - self.A0 @ u_prev))

    @property
    def sizes(self):
        return [self.A0.shape[0]] + [lev.A.shape[0] for lev in self.levels]
