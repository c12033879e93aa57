"""Pins of the oracle's multiscale multigrid (Sec. 3) against facts fixed by
the method's definition and by linear algebra:

* node partition (each free node in exactly one block);
* Eq. (8): the internal Neumann matrices annihilate constants and are SPSD;
  the basis is M-orthonormal, satisfies the generalised eigen-equation, and
  with L = 1 reduces to the kappa-mass-normalised block indicator;
* Eq. (9): mass = identity on every group ("mass trick"), orthonormal Psi,
  the group's constant function stays in the coarse-coarse space;
* complete local bases make the V-cycle an exact solver (two- and three-grid);
* the algorithmic V-cycle (Algorithm 1) equals its closed product form built
  here from dense matrices, is symmetric and positive definite;
* the coarse initial guess is Galerkin-orthogonal: P^T (b - A u0) = 0;
* MMG-PCG reproduces a direct solve;
* the l1-block-Jacobi smoother: D_l1 - A is SPSD, so the spectrum of
  D_l1^-1 A lies in (0, 1].
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fem, krylov, mmg


def _prob(N=8, seed=5, kmin=1e-3, density="rand", mask=None):
    grid = (N, N, N)
    if density == "rand":
        x = W.uniform01(seed, N ** 3)
    elif density == "chan":
        x = W.channel_tree_density(N, seed, 0.2)
    else:
        x = np.full(N ** 3, 0.5)
    m = W.dirichlet_patch_mask(grid) if mask is None else mask
    return fem.build_problem(grid, (1.0 / N,) * 3, x, 3.0, kmin, 1.0, m, W.uniform_source(grid))


def test_node_partition_is_disjoint_cover():
    P = _prob(N=8)
    blk, shape = mmg.node_blocks(P["grid"], 4, P["mask"])
    assert shape == (2, 2, 2)
    free = ~P["mask"]
    assert np.all(blk[free] >= 0) and np.all(blk[~free] == -1)
    cnt = np.bincount(blk[free], minlength=8)
    # last block of each axis takes the closing plane: 4 or 5 planes per axis
    sizes = sorted(set(cnt.tolist()))
    assert cnt.sum() == free.sum()
    assert sizes[-1] <= 125 and sizes[0] >= 64 - 9


def test_local_neumann_and_mass_normalisation():
    P = _prob(N=8)
    o = mmg.MMGOptions(block=4, nvec=(4,), group=())
    P1, act, eigs, blk, shape = mmg.level1_basis(P, o)
    A = P["A"].tocsr()
    m = P["mass"]
    # sum_i m_i over all nodes = int kappa dV (kappa-weighted lumped mass)
    assert abs(m.sum() - P["kappa"].sum() / 8 ** 3) < 1e-13
    P1d = P1.toarray()
    for c in range(8):
        idx = np.flatnonzero(blk == c)
        ABB = A[idx][:, idx].toarray()
        At = ABB - np.diag(ABB.sum(axis=1))
        assert np.max(np.abs(At @ np.ones(idx.size))) < 1e-14 * np.abs(At).max()
        assert np.linalg.eigvalsh(At)[0] > -1e-13 * np.abs(At).max()
        Phi = P1d[idx][:, c * 4:(c + 1) * 4]
        G = Phi.T @ (m[idx][:, None] * Phi)
        np.testing.assert_allclose(G, np.eye(4), atol=1e-13)
        lam = eigs[c]
        R = At @ Phi - (m[idx][:, None] * Phi) * lam[None, :]
        assert np.abs(R).max() <= 1e-10 * np.abs(At).max()
        assert abs(lam[0]) < 1e-10 * np.abs(At).max() / m[idx].min()
        # first vector: constant on the block (null space of the Neumann form)
        ph0 = Phi[:, 0]
        np.testing.assert_allclose(ph0, ph0.mean(), rtol=1e-8)


def test_single_vector_is_normalised_block_indicator():
    P = _prob(N=8, seed=9)
    o = mmg.MMGOptions(block=4, nvec=(1,), group=())
    P1, _, _, blk, _ = mmg.level1_basis(P, o)
    m = P["mass"]
    for c in range(8):
        idx = np.flatnonzero(blk == c)
        want = 1.0 / np.sqrt(m[idx].sum())
        np.testing.assert_allclose(P1[idx, c].toarray().ravel(), want, rtol=1e-12)


def test_coarse_coarse_mass_is_identity_and_constants_preserved():
    P = _prob(N=16, seed=4)
    o = mmg.MMGOptions(block=4, nvec=(4, 8), group=(2,))
    H = mmg.MMG(P, o)
    Pc = H.Pcomp.toarray()                        # fine <- level 2
    G = Pc.T @ (P["mass"][:, None] * Pc)
    np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-12)
    Psi = H.levels[1].P.toarray()
    np.testing.assert_allclose(Psi.T @ Psi, np.eye(Psi.shape[1]), atol=1e-12)
    # the indicator of every group (on free nodes) lies in range(Pc)
    blk, _ = mmg.node_blocks(P["grid"], 4, P["mask"])
    bx = blk % 4
    by = (blk // 4) % 4
    bz = blk // 16
    grp = (bx // 2) + 2 * ((by // 2) + 2 * (bz // 2))
    for g in range(8):
        ind = ((grp == g) & (blk >= 0)).astype(float)
        coef = np.linalg.lstsq(Pc, ind, rcond=None)[0]
        assert np.linalg.norm(Pc @ coef - ind) < 1e-9 * np.linalg.norm(ind)


def _free_random(P, seed):
    r = W.uniform01(seed, P["A"].shape[0]) - 0.5
    r[P["mask"]] = 0.0
    return r


def test_complete_local_basis_gives_exact_two_grid():
    P = _prob(N=4, seed=3)
    o = mmg.MMGOptions(block=2, nvec=(27,), group=())
    H = mmg.MMG(P, o)
    r = _free_random(P, 1)
    e = H(r)
    exact = spla.spsolve(P["A"].tocsc(), r)
    np.testing.assert_allclose(e, exact, rtol=1e-9, atol=1e-11 * np.abs(exact).max())


def test_complete_bases_give_exact_three_grid():
    P = _prob(N=8, seed=3)
    o = mmg.MMGOptions(block=2, nvec=(27, 216), group=(2,))
    H = mmg.MMG(P, o)
    r = _free_random(P, 2)
    e = H(r)
    exact = spla.spsolve(P["A"].tocsc(), r)
    np.testing.assert_allclose(e, exact, rtol=1e-8, atol=1e-10 * np.abs(exact).max())


def _dense_vcycle_matrix(H, P):
    """Closed product form of the V-cycle: B = (I - E) A^{-1} with
    E = S^nu (I - P B_c P^T A) S^nu, S = I - W^{-1} A (W the smoother),
    B_c the coarse V-cycle (recursively) or A_L^{-1} at the coarsest grid."""
    o = H.opts
    mats = [P["A"].toarray()] + [lev.A.toarray() for lev in H.levels]
    Ps = [lev.P.toarray() for lev in H.levels]

    def smoother_inv(l):
        A = mats[l]
        if l == 0:
            return o.omega * np.diag(1.0 / np.diag(A))
        L = H.levels[l - 1].L
        n = A.shape[0]
        Winv = np.zeros((n, n))
        for c in range(n // L):
            s = slice(c * L, (c + 1) * L)
            D = A[s, s].copy()
            off = np.abs(A[s]).sum(axis=1) - np.abs(A[s, s]).sum(axis=1)
            Winv[s, s] = np.linalg.inv(D + np.diag(off))
        return Winv

    def B(l):
        A = mats[l]
        if l == len(mats) - 1:
            return np.linalg.inv(A)
        nu = o.nu_fine if l == 0 else min(64, o.nu_coarse * o.nu_growth ** (l - 1))
        I = np.eye(A.shape[0])
        S = I - smoother_inv(l) @ A
        Sn = np.linalg.matrix_power(S, nu)
        # coarse corrections per visit: two (W-cycle) on levels >= w_from above the second-coarsest
        reps = 2 if (l >= 1 and o.w_from > 0 and l >= o.w_from and l + 2 < len(mats)) else 1
        C = np.linalg.matrix_power(I - Ps[l] @ B(l + 1) @ Ps[l].T @ A, reps)
        E = Sn @ C @ Sn
        return (I - E) @ np.linalg.inv(A)

    return B(0)


def test_vcycle_equals_closed_product_form():
    P = _prob(N=8, seed=21)
    o = mmg.MMGOptions(block=2, nvec=(4, 6), group=(2,))
    H = mmg.MMG(P, o)
    Bd = _dense_vcycle_matrix(H, P)
    n = P["A"].shape[0]
    rng_cols = [0, 5, 100, 333, n - 1]
    for j in rng_cols:
        ej = np.zeros(n)
        ej[j] = 1.0
        np.testing.assert_allclose(H(ej), Bd[:, j], rtol=1e-9, atol=1e-12 * np.abs(Bd).max())


def test_wcycle_with_growing_sweeps_equals_closed_product_form():
    """Three coarse levels, sweeps doubling per level and two coarse
    corrections per visit on level 1: the recursive cycle equals the dense
    product form E_l = S^nu_l (I - P B_(l+1) P^T A)^2 S^nu_l, and stays
    symmetric positive definite."""
    P = _prob(N=8, seed=23)
    o = mmg.MMGOptions(block=2, nvec=(4, 6, 6), group=(2, 2), nu_growth=2, w_from=1)
    H = mmg.MMG(P, o)
    assert len(H.levels) == 3
    Bd = _dense_vcycle_matrix(H, P)
    n = P["A"].shape[0]
    for j in [0, 9, 200, n - 1]:
        ej = np.zeros(n)
        ej[j] = 1.0
        np.testing.assert_allclose(H(ej), Bd[:, j], rtol=1e-9, atol=1e-12 * np.abs(Bd).max())
    x = _free_random(P, 3)
    y = _free_random(P, 4)
    assert abs(H(x) @ y - x @ H(y)) <= 1e-12 * np.linalg.norm(H(x)) * np.linalg.norm(y)
    assert x @ H(x) > 0
    # the W-cycle is a better solver than the V-cycle on the same hierarchy
    ov = mmg.MMGOptions(block=2, nvec=(4, 6, 6), group=(2, 2), nu_growth=1, w_from=0)
    Bv = _dense_vcycle_matrix(mmg.MMG(P, ov), P)
    A = P["A"].toarray()
    free = ~P["mask"]
    I = np.eye(n)
    rho = lambda B: np.abs(np.linalg.eigvals((I - B @ A)[np.ix_(free, free)])).max()
    assert rho(Bd) < rho(Bv)


def test_vcycle_symmetric_positive_definite():
    P = _prob(N=16, seed=8, density="chan", kmin=1e-6)
    H = mmg.MMG(P)
    x = _free_random(P, 11)
    y = _free_random(P, 12)
    Bx, By = H(x), H(y)
    assert abs(Bx @ y - x @ By) <= 1e-12 * np.linalg.norm(Bx) * np.linalg.norm(y)
    assert x @ Bx > 0 and y @ By > 0


def test_coarse_initial_guess_is_galerkin_orthogonal():
    P = _prob(N=16, seed=6)
    H = mmg.MMG(P)
    u0 = H.coarse_guess(P["b"])
    res = H.Pcomp.T @ (P["b"] - P["A"] @ u0)
    assert np.abs(res).max() <= 1e-12 * np.abs(H.Pcomp.T @ P["b"]).max()
    u1 = H.coarse_guess(P["b"], u_prev=0.5 * u0 + 0.01)
    res1 = H.Pcomp.T @ (P["b"] - P["A"] @ u1)
    assert np.abs(res1).max() <= 1e-11 * np.abs(H.Pcomp.T @ P["b"]).max()


@pytest.mark.parametrize("density,kmin", [("rand", 1e-3), ("chan", 1e-6)])
def test_mmg_pcg_matches_direct_solve(density, kmin):
    P = _prob(N=16, seed=2, density=density, kmin=kmin)
    H = mmg.MMG(P)
    u, info = krylov.pcg(P["A"], P["b"], precond=H, u0=H.coarse_guess(P["b"]), tol=1e-12)
    assert info["converged"], info["iters"]
    ud = spla.spsolve(P["A"].tocsc(), P["b"])
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
    # a robust preconditioner: far fewer iterations than Jacobi-PCG
    _, ij = krylov.pcg(P["A"], P["b"], precond=krylov.jacobi_precond(P["A"]), tol=1e-12,
                       maxit=20000)
    assert info["iters"] * 3 < ij["iters"]


def _cheb_poly(lam, lo, hi, m):
    """Scaled Chebyshev polynomial T_m((hi+lo-2 lam)/(hi-lo)) / T_m((hi+lo)/(hi-lo))."""
    def T(x):
        x = np.asarray(x, float)
        out = np.empty_like(x)
        inside = np.abs(x) <= 1
        out[inside] = np.cos(m * np.arccos(x[inside]))
        xo = x[~inside]
        out[~inside] = np.sign(xo) ** m * np.cosh(m * np.arccosh(np.abs(xo)))
        return out
    return T((hi + lo - 2 * lam) / (hi - lo)) / T(np.array([(hi + lo) / (hi - lo)]))[0]


def test_lmax_estimate_below_and_close_to_true():
    P = _prob(N=6, seed=12, kmin=1e-4)
    A = P["A"].toarray()
    D = np.diag(A)
    free = ~P["mask"]
    Af = A[np.ix_(free, free)]
    Df = D[free]
    lam_true = np.linalg.eigvalsh(Af / np.sqrt(Df)[:, None] / np.sqrt(Df)[None, :]).max()
    est = mmg.lmax_estimate(P["A"], D, free.astype(float), 15)
    assert est <= lam_true * (1 + 1e-12)
    assert est >= 0.85 * lam_true


@pytest.mark.parametrize("N", [16, 32])
def test_lmax_estimate_covers_the_spectrum_on_uniform_media(N):
    """Uniform conductivity: the top of the spectrum of D^-1 A is a dense cluster
    at 3/2 (cubic Q1: the mode alternating along one axis).  From the seeded
    start vector, 15 power iterations come within 7% of it, so the Chebyshev
    interval's upper end 1.1 lmax covers the spectrum."""
    import scipy.sparse as sp
    grid = (N, N, N)
    P = fem.build_problem(grid, (1.0 / N,) * 3, np.full(N ** 3, 0.3), 3.0, 1e-3, 1.0,
                          W.dirichlet_patch_mask(grid), W.uniform_source(grid))
    A = P["A"].tocsr()
    D = A.diagonal()
    free = (~P["mask"]).astype(float)
    Dm = sp.diags(1 / np.sqrt(D))
    lam_true = spla.eigsh(Dm @ A @ Dm, k=1, which="LA", return_eigenvectors=False)[0]
    assert abs(lam_true - 1.5) < 1e-3
    est = mmg.lmax_estimate(A, D, free, 15)
    assert 0.93 * lam_true <= est <= lam_true * (1 + 1e-12)
    assert 1.1 * est >= lam_true


def test_mmg_pcg_converges_on_uniform_media():
    """Regression: on a uniform density the multigrid-preconditioned CG converges
    as fast as on a random one (an underestimated lmax made it stall)."""
    N = 32
    grid = (N, N, N)
    P = fem.build_problem(grid, (1.0 / N,) * 3, np.full(N ** 3, 0.3), 3.0, 1e-3, 1.0,
                          W.dirichlet_patch_mask(grid), W.uniform_source(grid))
    H = mmg.MMG(P)
    _, info = krylov.pcg(P["A"], P["b"], precond=H, u0=H.coarse_guess(P["b"]), tol=1e-8, maxit=200)
    assert info["converged"] and info["iters"] <= 30, info["iters"]


@pytest.mark.parametrize("m", [2, 3, 4])
def test_chebyshev_smoother_is_scaled_chebyshev_polynomial(m):
    """The smoother's error propagation (r = A e*, start e = 0, error e* - e)
    equals p(D^-1 A) with p the scaled Chebyshev polynomial on [lo, hi]."""
    P = _prob(N=4, seed=13, kmin=1e-3)
    o = mmg.MMGOptions(block=2, nvec=(4,), group=(), smoother="chebyshev", cheb_degree=m)
    H = mmg.MMG(P, o)
    A = P["A"].toarray()
    D = np.diag(A)
    free = ~P["mask"]
    Af = A[np.ix_(free, free)]
    s = 1 / np.sqrt(D[free])
    lam, V = np.linalg.eigh(Af * s[:, None] * s[None, :])
    lo, hi = H.lmax / 30.0, 1.1 * H.lmax
    p = _cheb_poly(lam, lo, hi, m)
    Efree = (s[:, None] * V) @ np.diag(p) @ (V.T / s[None, :])   # D^-1/2 p(C) D^1/2
    n = A.shape[0]
    idx = np.flatnonzero(free)
    for j in [0, 7, len(idx) - 1]:
        estar = np.zeros(n)
        estar[idx[j]] = 1.0
        e = H._chebyshev(A @ estar, np.zeros(n))
        np.testing.assert_allclose((estar - e)[free], Efree[:, j], atol=1e-12)


def test_vcycle_closed_form_with_chebyshev():
    P = _prob(N=8, seed=22)
    o = mmg.MMGOptions(block=2, nvec=(4, 6), group=(2,), smoother="chebyshev", cheb_degree=3)
    H = mmg.MMG(P, o)
    A = P["A"].toarray()
    D = np.diag(A)
    free = ~P["mask"]
    s = 1 / np.sqrt(D)
    lam, V = np.linalg.eigh(A * s[:, None] * s[None, :])
    lo, hi = H.lmax / 30.0, 1.1 * H.lmax
    Sfine = (s[:, None] * V) @ np.diag(_cheb_poly(lam, lo, hi, 3)) @ (V.T / s[None, :])
    mats = [lev.A.toarray() for lev in H.levels]
    Ps = [lev.P.toarray() for lev in H.levels]
    L = H.levels[0].L
    A1 = mats[0]
    W1 = np.zeros_like(A1)
    for c in range(A1.shape[0] // L):
        sl = slice(c * L, (c + 1) * L)
        off = np.abs(A1[sl]).sum(axis=1) - np.abs(A1[sl, sl]).sum(axis=1)
        W1[sl, sl] = np.linalg.inv(A1[sl, sl] + np.diag(off))
    I1 = np.eye(A1.shape[0])
    S1 = I1 - W1 @ A1
    E1 = S1 @ (I1 - Ps[1] @ np.linalg.inv(mats[1]) @ Ps[1].T @ A1) @ S1
    B1 = (I1 - E1) @ np.linalg.inv(A1)
    # Dirichlet rows are identities; the smoother leaves them at zero
    Sf = np.where(free[:, None] & free[None, :], Sfine, 0.0)
    I = np.eye(A.shape[0])
    Sf = Sf + np.diag((~free).astype(float)) * 0.0
    E = Sf @ (I - Ps[0] @ B1 @ Ps[0].T @ A) @ Sf
    Ainv = np.linalg.inv(A)
    B = (I - E) @ Ainv
    for j in np.flatnonzero(free)[[0, 11, 100, -1]]:
        ej = np.zeros(A.shape[0])
        ej[j] = 1.0
        np.testing.assert_allclose(H(ej)[free], B[free, j], rtol=1e-9, atol=1e-12 * np.abs(B).max())


def test_l1_block_jacobi_is_convergent_without_damping():
    """The l1-block-Jacobi smoother of the coarse levels (Baker, Falgout, Kolev
    and Yang, 2011): D_l1 = A_cc + diag(sum of the off-cell |a_ij|) makes
    D_l1 - A symmetric positive semidefinite (a symmetric diagonally dominant
    matrix with a nonnegative diagonal), so the spectrum of D_l1^-1 A lies in
    (0, 1] and one undamped sweep reduces the error in the A-norm.  With no
    off-cell couplings (one cell) D_l1 = A and the sweep is exact."""
    P = _prob(N=16, density="chan", kmin=1e-6)
    H = mmg.MMG(P, mmg.MMGOptions(block=4, nvec=(4, 17), group=(2,), smoother="chebyshev"))
    lev = H.levels[0]
    A = lev.A.toarray()
    L = lev.L
    D = np.zeros_like(A)
    for c, Dinv in enumerate(lev.smoother):
        s = slice(c * L, (c + 1) * L)
        D[s, s] = np.linalg.inv(Dinv)
    act = np.flatnonzero(lev.active)
    A, D = A[np.ix_(act, act)], D[np.ix_(act, act)]
    assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
    assert np.linalg.eigvalsh(D - A).min() >= -1e-12 * np.abs(A).max()
    ev = np.linalg.eigvals(np.linalg.solve(D, A)).real
    assert ev.min() > 0.0 and ev.max() <= 1.0 + 1e-10
    # a single cell: the l1 block is the whole operator
    one = mmg.l1_block_inverses(lev.A[:L, :L], (1, 1, 1), L)[0]
    np.testing.assert_allclose(one @ lev.A[:L, :L].toarray(), np.eye(L), atol=1e-10)


def test_given_bases_reproduce_the_computed_hierarchy():
    """MMG(..., bases=the oracle's own prolongations) is the same preconditioner:
    identical Galerkin operators, cycle and coarse guess (the hook that lets a
    test evaluate the cycle on the library's exported bases)."""
    import workloads as W
    pr = W.problem("chan32")
    P = fem.build_problem(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], pr["mask"],
                          pr["source"])
    H = mmg.MMG(P)
    G = mmg.MMG(P, bases=[lev.P for lev in H.levels])
    for a, b in zip(H.levels, G.levels):
        assert (a.A != b.A).nnz == 0
        assert np.array_equal(a.active, b.active)
    r = np.random.default_rng(5).standard_normal(P["A"].shape[0])
    r[P["mask"]] = 0.0
    assert np.array_equal(H(r), G(r))
    assert np.array_equal(H.coarse_guess(P["b"]), G.coarse_guess(P["b"]))


def _inclusions_problem(kmin=1e-6):
    """8^3 grid, blocks of 4^3: three single-element solid inclusions (x = 1)
    that share no node, inside block 0, in void (x = 0) elsewhere; the
    Dirichlet patch node lies in another block."""
    N = 8
    x = np.zeros((N, N, N))
    for (ex, ey, ez) in [(0, 0, 0), (2, 0, 0), (0, 2, 2)]:
        x[ez, ey, ex] = 1.0
    grid = (N, N, N)
    return fem.build_problem(grid, (1.0 / N,) * 3, x.ravel(), 3.0, kmin, 1.0, W.dirichlet_patch_mask(grid),
                             W.uniform_source(grid))


def test_adaptive_count_equals_high_conductivity_components():
    """Adaptive local bases (eig_threshold tau): in a high-contrast block the
    kappa-weighted Neumann problem has one eigenvalue near zero per
    high-conductivity component (in the kappa-mass norm the constant is the sum
    of their indicators: void-supported functions carry almost no mass), the
    rest above about 1 / h^2.  So tau = 1 (a threshold 1 / H^2) keeps exactly
    one vector per inclusion in block 0 and one (the constant) in the void
    blocks -- fixed by the spectrum, checked against numpy's eigenvalues of
    each block's dense problem."""
    P = _inclusions_problem()
    o = mmg.MMGOptions(block=4, nvec=(6,), group=(), eig_threshold=1.0)
    P1, act, eigs, blk, shape = mmg.level1_basis(P, o)
    counts = act.reshape(-1, 6).sum(axis=1)
    assert counts[0] == 3, counts
    assert np.all(counts[1:] == 1), counts
    H = 4 * (1.0 / 8)
    # the spectrum behind the count: three tiny eigenvalues in block 0, then a gap
    w0 = eigs[0]
    assert np.all(w0[:3] * H ** 2 < 1e-3) and len(w0) == 3
    full = mmg.level1_basis(P, mmg.MMGOptions(block=4, nvec=(6,), group=()))[2][0]
    assert full[3] * H ** 2 > 1.0, full


def test_adaptive_with_a_huge_threshold_is_the_fixed_hierarchy():
    """tau above every local eigenvalue keeps nvec vectors everywhere: the same
    preconditioner as the fixed counts (bases, operators, cycle)."""
    pr = W.problem("chan32")
    P = fem.build_problem(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], pr["mask"],
                          pr["source"])
    o0 = mmg.default_options(32)
    o1 = mmg.default_options(32)
    o1.eig_threshold = 1e300
    H0, H1 = mmg.MMG(P, o0), mmg.MMG(P, o1)
    for a, b in zip(H0.levels, H1.levels):
        assert np.array_equal(a.active, b.active)
        assert (a.A != b.A).nnz == 0
    r = np.random.default_rng(7).standard_normal(P["A"].shape[0])
    r[P["mask"]] = 0.0
    assert np.array_equal(H0(r), H1(r))


def test_adaptive_hierarchy_preconditions_cg():
    """A moderate threshold gives a smaller coarse space that still makes
    MMG-PCG reproduce the direct solve."""
    pr = W.problem("chan32")
    P = fem.build_problem(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], pr["mask"],
                          pr["source"])
    o = mmg.default_options(32)
    o.eig_threshold = 2.0
    H = mmg.MMG(P, o)
    kept = [int(l.active.sum()) for l in H.levels]
    full = [l.active.size for l in H.levels]
    assert kept[0] < full[0]
    free = ~P["mask"]
    u, info = krylov.pcg(P["A"], P["b"], precond=H, u0=H.coarse_guess(P["b"]), tol=1e-10, free=free)
    ud = spla.spsolve(P["A"].tocsc(), P["b"])
    assert info["converged"] and np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud), info


def test_sign_convention():
    """R13: the entry of largest magnitude (lowest index on ties) is positive."""
    v = np.array([0.1, -0.7, 0.7, 0.2])
    np.testing.assert_array_equal(mmg._sign_fix(v), -v)  # tie: index 1 wins, it is negative
    w = np.array([0.1, 0.3, -0.2])
    np.testing.assert_array_equal(mmg._sign_fix(w), w)
    np.testing.assert_array_equal(mmg._sign_fix(-w), w)
