"""Pins of the oracle's TPFA discretisation (oracle/tpfa.py: the paper's
cell-centred scheme of Sec. 2.2, the design-dependent source of Sec. 2.1 and
the mean-temperature adjoint of Sec. 2.3) against facts fixed by the
mathematics, not by re-typing its formulas:

* symmetry; zero row sums without Dirichlet faces; positive definiteness with
  them;
* exactness in 1-D series conduction (layered conductivity between two
  Dirichlet faces, no source): the cell-centre temperatures lie on the exact
  piecewise-linear profile, which fixes the harmonic face mean and the
  half-cell Dirichlet transmissibility;
* second-order convergence at the cell centres on a manufactured solution;
* the adjoint identity c = u^T b, and the sensitivity against exact central
  differences of the mean temperature (every term: faces, Dirichlet faces,
  source).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import tpfa


def _prob(grid, x, kmin=1e-2, face="z0_full", TD=0.0, f0=1.0, p=3.0, source=None):
    h = tuple(1.0 / g for g in grid)
    return tpfa.build(grid, h, x, p, kmin, 1.0, f0, tpfa.dirichlet_faces(grid, face), TD=TD, source=source)


def test_operator_symmetric_conservative_spd():
    grid = (4, 3, 5)
    M = 60
    x = W.uniform01(81, M)
    P = _prob(grid, x)
    A = P["A"].toarray()
    assert np.allclose(A, A.T, rtol=0, atol=1e-15 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    # without Dirichlet faces the operator is the all-Neumann one: rows sum to zero
    N = tpfa.build(grid, tuple(1.0 / g for g in grid), x, 3.0, 1e-2, 1.0, 1.0, {})["A"].toarray()
    assert np.max(np.abs(N.sum(axis=1))) <= 1e-14 * np.abs(N).max()
    # off-diagonal entries are -kappa_F |F| / h with the harmonic mean (cells 0 and 1 share an x face)
    k = P["kappa"]
    hx, hy, hz = 1 / 4, 1 / 3, 1 / 5
    assert abs(-A[0, 1] - 2 / (1 / k[0] + 1 / k[1]) * hy * hz / hx) <= 1e-15 * abs(A[0, 1])


@pytest.mark.parametrize("N", [3, 8])
def test_series_conduction_is_exact(N):
    """Layers of conductivity k_z between T = 0 at z = 0 and T = 1 at z = 1, no
    source: the exact temperature at height s is R(s) / R(1) with the thermal
    resistance R(s) = int_0^s dz / k(z)."""
    grid = (2, 3, N)
    kz = 10.0 ** np.linspace(-6, 0, N)[np.random.default_rng(N).permutation(N)]
    x = np.repeat(kz, 6)  # with p = 1, kmin = 0, kmax = 1: kappa = x
    P = tpfa.build(grid, (0.5, 1 / 3, 1.0 / N), x, 1.0, 0.0, 1.0, 0.0,
                   tpfa.dirichlet_faces(grid, "z0z1_full"), TD={(2, 0): 0.0, (2, 1): 1.0})
    t = spla.spsolve(P["A"].tocsc(), P["b"])
    h = 1.0 / N
    R_centre = np.cumsum(h / kz) - 0.5 * h / kz      # resistance from z = 0 to each layer's centre
    exact = np.repeat(R_centre / np.sum(h / kz), 6)
    np.testing.assert_allclose(t, exact, rtol=1e-9, atol=1e-12)


def test_manufactured_solution_second_order():
    """T = cos(pi x) cos(pi y) z (2 - z): T = 0 on z = 0, no normal flux on the
    other faces; kappa = 1, f = -Lap T sampled at the cell centres."""
    errs = []
    for N in (8, 16, 32):
        grid = (N, N, N)
        c = (np.arange(N) + 0.5) / N
        zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
        T = np.cos(np.pi * xx) * np.cos(np.pi * yy) * zz * (2 - zz)
        f = np.cos(np.pi * xx) * np.cos(np.pi * yy) * (2 * np.pi ** 2 * zz * (2 - zz) + 2.0)
        P = _prob(grid, np.ones(N ** 3), source=f.ravel())
        t = spla.spsolve(P["A"].tocsc(), P["b"])
        errs.append(np.max(np.abs(t - T.ravel())))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


def _solve(P):
    return spla.spsolve(P["A"].tocsc(), P["b"])


@pytest.mark.parametrize("face,TD", [("z0_full", 0.0), ("z0", 100.0)])
def test_adjoint_identity_and_central_differences(face, TD):
    grid = (4, 4, 6) if face == "z0_full" else (10, 10, 4)
    M = grid[0] * grid[1] * grid[2]
    x = 0.2 + 0.8 * W.uniform01(82, M)
    P = _prob(grid, x, face=face, TD=TD)
    assert any(m.any() for m in P["dfaces"].values())
    t = _solve(P)
    c = tpfa.mean_temperature(t)
    u = spla.spsolve(P["A"].tocsc(), tpfa.adjoint_rhs(M))
    assert abs(u @ P["b"] - c) <= 1e-12 * abs(c)
    g = tpfa.sensitivity(P, t, u)
    for e in [0, 7, M // 2, M - 1]:
        # central differences of c formed without cancellation: c(x') - c(x) is the mean of
        # t' - t = A'^-1 (b' - A' t), whose right-hand side involves only the changed entries
        d = 1e-5
        dc = []
        for s in (+1, -1):
            xe = x.copy()
            xe[e] += s * d
            Q = _prob(grid, xe, face=face, TD=TD)
            dt = spla.spsolve(Q["A"].tocsc(), Q["b"] - Q["A"] @ t)
            dc.append(dt.mean())
        fd = (dc[0] - dc[1]) / (2 * d)
        assert abs(fd - g[e]) <= 1e-6 * abs(g[e]), (e, fd, g[e])


@pytest.mark.parametrize("N,kmin", [(16, 1e-3), (16, 1e-6), (16, 1e-9), (32, 1e-6)])
def test_mmg_on_the_tpfa_system_reproduces_the_direct_solve(N, kmin):
    """The algebraic construction of Sec. 3 (oracle.mmg on the cells' b^3
    blocks, kappa-weighted cell mass, the same cycle) preconditions the paper's
    own TPFA system: MMG-PCG from the coarse guess reaches the direct solution,
    in a number of iterations that does not grow with the contrast (10-13 for
    contrasts 1e3-1e9 on the channel design)."""
    from oracle import krylov, mmg
    grid = (N, N, N)
    x = W.channel_tree_density(N, 3, 0.2)
    P = tpfa.build(grid, (1.0 / N,) * 3, x, 3.0, kmin, 1.0, 1.0, tpfa.dirichlet_faces(grid, "z0"))
    Q = tpfa.mmg_problem(P)
    H = mmg.MMG(Q, mmg.default_options(N))
    u, info = krylov.pcg(Q["A"], Q["b"], precond=H, u0=H.coarse_guess(Q["b"]), tol=1e-10, free=~Q["mask"])
    ud = spla.spsolve(Q["A"].tocsc(), Q["b"])
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud), info
    assert info["iters"] <= 20, info
