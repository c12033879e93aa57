"""Preconditioner set-up on the GPU (Sec. 3, Eqs. (8)-(9)) checked against
the oracle and against the properties the construction must satisfy:
M-orthonormal level-1 bases that solve the local generalised eigenproblem,
the same spanned subspaces as the oracle where the eigengap is clear,
Galerkin tiles equal to Phi^T A Phi, orthonormal Psi, and the coarsest
inverse."""
import numpy as np
import pytest
import scipy.sparse as sp

from helpers import gpu_solver, oracle_problem, small_problem
from oracle import mmg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup16():
    pr = small_problem(16, kind="smooth")
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=0)
    s.setup_precond()
    H = mmg.MMG(P)
    yield pr, P, s, H
    s.close()


def _phi_gpu(s, P):
    n = P["A"].shape[0]
    return s.export_level(1, 0, n * 4).cpu().numpy().reshape(n, 4)


def test_level1_basis_mass_orthonormal_and_eigen(setup16):
    pr, P, s, H = setup16
    phi = _phi_gpu(s, P)
    blk, shape = mmg.node_blocks(pr["grid"], 4, pr["mask"])
    A = P["A"].tocsr()
    m = P["mass"]
    eig = s.export_level(1, 2, 64 * 4).cpu().numpy().reshape(64, 4)
    for c in range(64):
        idx = np.flatnonzero(blk == c)
        Phi = phi[idx]
        G = Phi.T @ (m[idx][:, None] * Phi)
        np.testing.assert_allclose(G, np.eye(4), atol=1e-12)
        ABB = A[idx][:, idx].toarray()
        At = ABB - np.diag(ABB.sum(axis=1))
        R = At @ Phi - (m[idx][:, None] * Phi) * eig[c][None, :]
        assert np.abs(R).max() <= 1e-4 * np.abs(At).max(), (c, np.abs(R).max())
        np.testing.assert_allclose(eig[c], H.levels[0].eigvals[c], rtol=1e-4, atol=1e-6 * np.abs(At).max() / m[idx].min())


def test_level1_subspaces_match_oracle(setup16):
    pr, P, s, H = setup16
    phi = _phi_gpu(s, P)
    blk, _ = mmg.node_blocks(pr["grid"], 4, pr["mask"])
    P1 = H.levels[0].P.toarray()
    m = P["mass"]
    for c in range(64):
        lam = H.levels[0].eigvals[c]
        idx = np.flatnonzero(blk == c)
        Po = P1[idx][:, c * 4:(c + 1) * 4]
        Pg = phi[idx]
        # M-orthogonal projectors onto the two spans
        Pro = Po @ Po.T * m[idx][None, :]
        Prg = Pg @ Pg.T * m[idx][None, :]
        assert np.abs(Pro - Prg).max() < 1e-4, c


def test_level1_galerkin_tiles_equal_phiT_A_phi(setup16):
    pr, P, s, H = setup16
    phi = _phi_gpu(s, P)
    n = P["A"].shape[0]
    T = s.export_level(1, 1, 64 * 27 * 16).cpu().numpy().reshape(64, 27, 4, 4)
    blk, _ = mmg.node_blocks(pr["grid"], 4, pr["mask"])
    rows, cols, vals = [], [], []
    for c in range(64):
        idx = np.flatnonzero(blk == c)
        for j in range(4):
            rows.append(idx)
            cols.append(np.full(idx.size, c * 4 + j))
            vals.append(phi[idx, j])
    Pg = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, 256))
    A1 = (Pg.T @ P["A"] @ Pg).toarray()
    full = np.zeros((256, 256))
    for c in range(64):
        cx, cy, cz = c % 4, (c // 4) % 4, c // 16
        for nn in range(27):
            dx, dy, dz = nn % 3 - 1, (nn // 3) % 3 - 1, nn // 9 - 1
            x2, y2, z2 = cx + dx, cy + dy, cz + dz
            if min(x2, y2, z2) < 0 or max(x2, y2, z2) > 3:
                assert np.abs(T[c, nn]).max() == 0.0
                continue
            c2 = x2 + 4 * (y2 + 4 * z2)
            full[c * 4:(c + 1) * 4, c2 * 4:(c2 + 1) * 4] = T[c, nn]
    np.testing.assert_allclose(full, A1, atol=1e-12 * np.abs(A1).max())


def test_coarsest_inverse_and_level2_orthonormal():
    pr = small_problem(32, kind="smooth")
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=0)
    s.setup_precond()
    hier = s.hierarchy()
    assert [h["ndof"] for h in hier] == [2048, 1088]
    psi = s.export_level(2, 0, 64 * 32 * 17).cpu().numpy().reshape(64, 32, 17)
    for G in range(64):
        np.testing.assert_allclose(psi[G].T @ psi[G], np.eye(17), atol=1e-12)
    T2 = s.export_level(2, 1, 64 * 27 * 17 * 17).cpu().numpy().reshape(64, 27, 17, 17)
    Ainv = s.export_level(2, 3, 1088 * 1088).cpu().numpy().reshape(1088, 1088)
    A2 = np.zeros((1088, 1088))
    for c in range(64):
        cx, cy, cz = c % 4, (c // 4) % 4, c // 16
        for nn in range(27):
            dx, dy, dz = nn % 3 - 1, (nn // 3) % 3 - 1, nn // 9 - 1
            x2, y2, z2 = cx + dx, cy + dy, cz + dz
            if min(x2, y2, z2) < 0 or max(x2, y2, z2) > 3:
                continue
            c2 = x2 + 4 * (y2 + 4 * z2)
            A2[c * 17:(c + 1) * 17, c2 * 17:(c2 + 1) * 17] = T2[c, nn]
    np.testing.assert_allclose(A2, A2.T, atol=1e-12 * np.abs(A2).max())
    np.testing.assert_allclose(Ainv @ A2, np.eye(1088), atol=1e-8)
    s.close()
