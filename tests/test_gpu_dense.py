"""The blocked FP64 Cholesky factorisation and explicit inverse of the direct
coarsest solve (Algorithm 1's A_cc^-1; a sparse LU in the paper's Sec. 4),
called on caller-supplied matrices through thermo_dense_spd_inverse:
inverses of SPD matrices against LAPACK's (numpy), orders that are and are
not multiples of the 64-wide tiles, and the THERMO_ESINGULAR path with the
exact index of the first non-positive pivot."""
import numpy as np
import pytest
import torch

from paper_2410_06850_gb300 import thermo

pytestmark = pytest.mark.gpu


def _spd(n, cond, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, np.log10(cond), n)
    return (Q * lam) @ Q.T


@pytest.mark.parametrize("n", [1, 63, 64, 100, 200, 1088])
def test_inverse_of_spd_matrices(n):
    A = _spd(n, 1e4, n)
    X, rc, piv, msg = thermo.dense_spd_inverse(torch.as_tensor(A).cuda())
    assert rc == thermo.OK, msg
    X = X.cpu().numpy()
    ref = np.linalg.inv(A)
    assert np.linalg.norm(X - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.linalg.norm(A @ X - np.eye(n)) <= 1e-10 * np.sqrt(n)
    assert np.array_equal(X, X.T)


@pytest.mark.parametrize("n,k", [(10, 0), (100, 37), (200, 130), (1088, 1087)])
def test_first_non_positive_pivot_is_reported(n, k):
    # diagonal matrix: the Cholesky pivots are the diagonal entries themselves
    d = np.linspace(1.0, 2.0, n)
    d[k] = -0.5
    if k + 3 < n:
        d[k + 3] = 0.0  # a later bad pivot must not replace the first
    X, rc, piv, msg = thermo.dense_spd_inverse(torch.as_tensor(np.diag(d)).cuda())
    assert rc == thermo.ESINGULAR and piv == k, (rc, piv, msg)


def test_indefinite_matrix_is_singular_status():
    A = _spd(150, 1e3, 7)
    w, V = np.linalg.eigh(A)
    w[0] = -1.0
    A = (V * w) @ V.T
    X, rc, piv, msg = thermo.dense_spd_inverse(torch.as_tensor(A).cuda())
    assert rc == thermo.ESINGULAR and 0 <= piv < 150, (rc, piv, msg)


def test_bad_arguments():
    X, rc, piv, msg = thermo.dense_spd_inverse(torch.zeros((0, 0), dtype=torch.float64, device="cuda"))
    assert rc == thermo.EINVAL
