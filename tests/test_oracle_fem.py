"""Pins of the FP64 oracle's discretisation against facts fixed by the
mathematics (not by re-typing the oracle's own formulas).

Q1 trilinear elements on box grids, SIMP conductivity (Sec. 2.1 Eq. (1)),
the Dirichlet-eliminated system of Sec. 2.2 Eq. (5), the compliance/mean
temperature of Eq. (6) and the adjoint sensitivity of Sec. 2.3.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fem


def _gauss_stiffness(h):
    """int grad(phi_a).grad(phi_b) over [0,hx]x[0,hy]x[0,hz] by 2-point Gauss
    per axis (exact: the integrand is at most quadratic per coordinate)."""
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    hx, hy, hz = h
    K = np.zeros((8, 8))
    for gx, gy, gz in itertools.product(g, g, g):
        s = np.array([(gx + 1) / 2, (gy + 1) / 2, (gz + 1) / 2])  # in [0,1]^3
        grads = []
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            fx = s[0] if ax else 1 - s[0]
            fy = s[1] if ay else 1 - s[1]
            fz = s[2] if az else 1 - s[2]
            dfx = (1 if ax else -1) / hx
            dfy = (1 if ay else -1) / hy
            dfz = (1 if az else -1) / hz
            grads.append([dfx * fy * fz, fx * dfy * fz, fx * fy * dfz])
        grads = np.array(grads)
        K += grads @ grads.T * (hx * hy * hz / 8.0)
    return K


@pytest.mark.parametrize("h", [(0.25, 0.25, 0.25), (0.3, 0.5, 0.7), (1.0, 2.0, 0.5)])
def test_element_matrix_matches_gauss_quadrature(h):
    np.testing.assert_allclose(fem.element_matrix(h), _gauss_stiffness(h),
                               rtol=1e-13, atol=1e-14)


def test_element_matrix_cube_closed_form():
    h = 0.125
    K = fem.element_matrix((h, h, h))
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            want = {0: h / 3, 1: 0.0, 2: -h / 12, 3: -h / 12}[d]
            assert abs(K[a, b] - want) < 1e-15
    ev = np.sort(np.linalg.eigvalsh(K))
    want = np.sort(h * np.array([0, 1 / 6, 1 / 3, 1 / 3, 1 / 3, 0.5, 0.5, 0.5]))
    np.testing.assert_allclose(ev, want, atol=1e-15)


def _small_problem(N=6, seed=11, mask="patch", kmin=1e-3):
    grid = (N, N, N)
    x = W.uniform01(seed, N ** 3)
    m = W.dirichlet_patch_mask(grid) if mask == "patch" else W.full_face_mask(grid, mask)
    return fem.build_problem(grid, (1.0 / N,) * 3, x, 3.0, kmin, 1.0, m, W.uniform_source(grid))


def test_operator_symmetric_spd_zero_rowsums_mmatrix():
    P = _small_problem()
    An = P["A_neu"].toarray()
    A = P["A"].toarray()
    assert np.array_equal(An, An.T)
    assert np.array_equal(A, A.T)
    assert np.max(np.abs(An.sum(axis=1))) <= 1e-15 * np.max(np.abs(An))
    np.linalg.cholesky(A)  # SPD after Dirichlet elimination
    assert np.min(np.linalg.eigvalsh(A)) > 0
    off = An - np.diag(np.diag(An))
    assert off.max() <= 1e-18  # cube Q1: couplings are non-positive (M-matrix)
    # all-Neumann operator is singular with the constants as kernel
    ev = np.linalg.eigvalsh(An)
    assert abs(ev[0]) < 1e-13 and ev[1] > 1e-8


def test_load_vector_integrates_source():
    N = 5
    grid = (N, N, N)
    q = 1.0 + W.uniform01(3, N ** 3)
    f = fem.load_vector(grid, (0.2, 0.2, 0.2), q)
    assert abs(f.sum() - q.sum() * 0.2 ** 3) < 1e-14


def test_dirichlet_count_of_patch():
    for N, cnt in [(32, 49), (128, 625), (256, 2601)]:
        assert int(W.dirichlet_patch_mask((N, N, N)).sum()) == cnt


def test_brute_force_dense_solve_matches_cg():
    from oracle import krylov
    P = _small_problem(N=5)
    u_dense = np.linalg.solve(P["A"].toarray(), P["b"])
    u, info = krylov.pcg(P["A"], P["b"], tol=1e-13)
    assert info["converged"]
    np.testing.assert_allclose(u, u_dense, rtol=1e-10, atol=1e-12 * np.abs(u_dense).max())


def _manufactured_error(N):
    grid = (N, N, N)
    h = 1.0 / N
    mask = W.full_face_mask(grid, "all")
    c = (np.arange(N) + 0.5) * h
    CZ, CY, CX = np.meshgrid(c, c, c, indexing="ij")
    q = (3 * np.pi ** 2 * np.sin(np.pi * CX) * np.sin(np.pi * CY) * np.sin(np.pi * CZ)).ravel()
    P = fem.build_problem(grid, (h, h, h), np.ones(N ** 3), 3.0, 1e-3, 1.0, mask, q)
    u = spla.spsolve(P["A"].tocsc(), P["b"])
    n = np.arange(N + 1) * h
    NZ, NY, NX = np.meshgrid(n, n, n, indexing="ij")
    ustar = (np.sin(np.pi * NX) * np.sin(np.pi * NY) * np.sin(np.pi * NZ)).ravel()
    return np.max(np.abs(u - ustar))


def test_manufactured_solution_second_order():
    errs = [_manufactured_error(N) for N in (8, 16, 32)]
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    for r in ratios:
        assert 3.6 < r < 4.4, (errs, ratios)


def test_exact_1d_solution_full_face_dirichlet():
    N = 8
    grid = (N, N, N)
    kap = 2.5
    P = fem.build_problem(grid, (1 / N,) * 3, np.ones(N ** 3), 3.0, 1e-3, kap,
                          W.full_face_mask(grid, "z0"), W.uniform_source(grid))
    u = spla.spsolve(P["A"].tocsc(), P["b"])
    z = (np.arange(N + 1) / N)[:, None, None] * np.ones((1, N + 1, N + 1))
    exact = ((z - z ** 2 / 2) / kap).ravel()
    np.testing.assert_allclose(u, exact, atol=1e-12)


@pytest.mark.parametrize("contrast", [1e0, 1e3, 1e6, 1e9])
def test_layered_exact_solution_high_contrast(contrast):
    N = 8
    grid = (N, N, N)
    k1, k2 = 1.0, 1.0 / contrast
    x = np.zeros((N, N, N))
    x[: N // 2] = 1.0  # elements with z < 1/2 are conductive
    mask = W.full_face_mask(grid, "z01")
    vals = np.zeros((N + 1, N + 1, N + 1))
    vals[-1] = 1.0
    P = fem.build_problem(grid, (1 / N,) * 3, x.ravel(), 1.0, k2, k1, mask,
                          np.zeros(N ** 3), values=vals.ravel())
    u = spla.spsolve(P["A"].tocsc(), P["b"])
    t = k2 / (k1 + k2)  # temperature at the interface (flux continuity)
    z = np.arange(N + 1) / N
    prof = np.where(z <= 0.5, t * z / 0.5, t + (1 - t) * (z - 0.5) / 0.5)
    exact = (prof[:, None, None] * np.ones((1, N + 1, N + 1))).ravel()
    np.testing.assert_allclose(u, exact, atol=1e-12)


def test_compliance_energy_identity_and_mean_temperature():
    P = _small_problem(N=6)
    u = spla.spsolve(P["A"].tocsc(), P["b"])
    c = fem.compliance(P["f"], u)
    assert abs(c - u @ (P["A"] @ u)) <= 1e-12 * abs(c)
    # f^T u = int u_h dV on the unit cube with q = 1 (trilinear quadrature exact)
    en = fem.element_nodes(P["grid"])
    integral = np.sum(u[en].mean(axis=1)) / 6 ** 3
    assert abs(c - integral) <= 1e-12 * abs(c)


def _solve(P):
    return spla.spsolve(P["A"].tocsc(), P["b"])


def test_sensitivity_euler_identity():
    P = _small_problem(N=6, kmin=0.05)
    u = _solve(P)
    c = fem.compliance(P["f"], u)
    dc = fem.sensitivity(P["grid"], P["h"], P["x"], 3.0, 0.05, 1.0, u)
    E = fem.element_energy(P["grid"], P["h"], u)
    lhs = np.sum(P["x"] * dc)
    rhs = -3.0 * (c - 0.05 * E.sum())
    assert abs(lhs - rhs) <= 1e-11 * abs(rhs)
    # kmin = 0 limit: c is homogeneous of degree -p in x
    P0 = _small_problem(N=6, kmin=0.0)
    P0["x"] = np.maximum(P0["x"], 0.05)
    P0 = fem.build_problem(P0["grid"], P0["h"], P0["x"], 3.0, 0.0, 1.0, P0["mask"],
                           W.uniform_source(P0["grid"]))
    u0 = _solve(P0)
    c0 = fem.compliance(P0["f"], u0)
    dc0 = fem.sensitivity(P0["grid"], P0["h"], P0["x"], 3.0, 0.0, 1.0, u0)
    assert abs(np.sum(P0["x"] * dc0) + 3.0 * c0) <= 1e-11 * c0


def test_sensitivity_central_finite_differences():
    P = _small_problem(N=5, kmin=0.01)
    u = _solve(P)
    dc = fem.sensitivity(P["grid"], P["h"], P["x"], 3.0, 0.01, 1.0, u)
    for e in [0, 17, 63, 124]:
        d = 1e-5
        xs = []
        for s in (+1, -1):
            x = P["x"].copy()
            x[e] += s * d
            Q = fem.build_problem(P["grid"], P["h"], x, 3.0, 0.01, 1.0, P["mask"],
                                  W.uniform_source(P["grid"]))
            xs.append(fem.compliance(Q["f"], _solve(Q)))
        fd = (xs[0] - xs[1]) / (2 * d)
        assert abs(fd - dc[e]) <= 1e-6 * abs(dc[e]) + 1e-14, (e, fd, dc[e])


@pytest.mark.parametrize("grid,h", [((8, 8, 8), (1 / 8,) * 3), ((6, 4, 5), (0.3, 0.5, 0.7))])
def test_row_evaluator_equals_assembled_operator(grid, h):
    """The unassembled row-by-row evaluation (used for full-size spot checks)
    equals the assembled Dirichlet-eliminated matrix (pinned above by its closed
    forms, symmetry, SPD and row sums) on every row, including identity rows
    and inputs that are nonzero on Gamma_D; its absolute variant gives |A||u|."""
    M = grid[0] * grid[1] * grid[2]
    x = W.uniform01(41, M)
    mask = W.dirichlet_patch_mask(grid)
    P = fem.build_problem(grid, h, x, 3.0, 1e-6, 1.0, mask, W.uniform_source(grid))
    n = P["A"].shape[0]
    u = W.uniform01(42, n) - 0.4
    rows = np.arange(n)
    y = fem.operator_rows(grid, h, P["kappa"], mask, u, rows, chunk=97)  # ragged chunks
    ref = P["A"] @ u
    scale = abs(P["A"]) @ np.abs(u)
    assert np.max(np.abs(y - ref) / scale) <= 1e-14
    ya = fem.operator_rows(grid, h, P["kappa"], mask, u, rows, absolute=True)
    np.testing.assert_allclose(ya, scale, rtol=1e-14, atol=0)
    sub = np.array([0, n - 1, n // 2, 17])
    np.testing.assert_array_equal(fem.operator_rows(grid, h, P["kappa"], mask, u, sub), y[sub])


@pytest.mark.parametrize("grid,h", [((8, 8, 8), (1 / 8,) * 3), ((6, 4, 5), (0.3, 0.5, 0.7))])
def test_sampled_load_and_sensitivity_equal_the_full_ones(grid, h):
    """The listed-nodes load (load_rows) and listed-elements sensitivity
    (sensitivity_at), used for spot checks of grids too large for whole
    vectors, equal load_vector (pinned by the integral of the source above)
    and sensitivity (pinned by the Euler identity and central differences)
    on every node and element, for a varying source and a scalar one."""
    M = grid[0] * grid[1] * grid[2]
    n = fem.n_nodes(grid)
    q = W.uniform01(43, M) + 0.5
    f = fem.load_vector(grid, h, q)
    np.testing.assert_allclose(fem.load_rows(grid, h, q, np.arange(n)), f, rtol=1e-15, atol=0)
    np.testing.assert_allclose(fem.load_rows(grid, h, 1.0, np.arange(n)),
                               fem.load_vector(grid, h, np.ones(M)), rtol=1e-15, atol=0)
    x = W.uniform01(44, M)
    u = W.uniform01(45, n) - 0.3
    dc = fem.sensitivity(grid, h, x, 3.0, 1e-3, 1.0, u)
    e = np.array([0, M - 1, M // 2, 5, 5])
    np.testing.assert_allclose(fem.sensitivity_at(grid, h, x[e], 3.0, 1e-3, 1.0, u, e), dc[e], rtol=1e-13, atol=0)
    np.testing.assert_allclose(fem.sensitivity_at(grid, h, x, 3.0, 1e-3, 1.0, u, np.arange(M)), dc,
                               rtol=1e-13, atol=1e-300)
