"""Pins of the oracle's conjugate-gradient solver (the outer iteration of
Sec. 4) by textbook properties of CG:

* with the exact inverse as preconditioner it converges in one iteration;
* without preconditioning it terminates after k iterations on an operator
  with k distinct eigenvalues;
* with a fixed SPD preconditioner the flexible (Polak-Ribiere) coefficient
  equals the standard one, because r_{k+1} is orthogonal to z_k, so both
  variants produce the same iterates (up to rounding);
* the A-norm of the error never grows from one iteration to the next.
"""
import numpy as np

import workloads as W
from oracle import krylov


def _spd(n, seed, cond=1e3):
    Q, _ = np.linalg.qr(W.uniform01(seed, n * n).reshape(n, n) - 0.5)
    lam = np.geomspace(1.0, cond, n)
    return (Q * lam) @ Q.T


def test_exact_preconditioner_converges_in_one_iteration():
    A = _spd(40, 71)
    b = W.uniform01(72, 40) - 0.5
    Ainv = np.linalg.inv(A)
    u, info = krylov.pcg(A, b, precond=lambda r: Ainv @ r, tol=1e-10)
    assert info["iters"] == 1 and info["converged"]
    np.testing.assert_allclose(u, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def test_terminates_after_as_many_iterations_as_distinct_eigenvalues():
    # the Krylov space of an operator with k distinct eigenvalues has dimension
    # at most k, so CG reaches the solution at iteration k
    n, k = 48, 4
    Q, _ = np.linalg.qr(W.uniform01(73, n * n).reshape(n, n) - 0.5)
    lam = np.repeat([1.0, 3.0, 7.0, 20.0], n // k)
    A = (Q * lam) @ Q.T
    b = W.uniform01(74, n) - 0.5
    u, info = krylov.pcg(A, b, tol=1e-11)
    assert info["converged"] and info["iters"] == k, info["iters"]
    assert info["history"][k - 1] > 1e-6  # not earlier


def test_flexible_equals_standard_with_a_fixed_preconditioner():
    n = 60
    A = _spd(n, 75, cond=1e2)
    b = W.uniform01(76, n) - 0.5
    d = 1.0 / (np.diag(A) * (1.0 + 0.5 * W.uniform01(77, n)))  # a fixed SPD (diagonal) preconditioner
    M = lambda r: d * r  # noqa: E731
    u0, i0 = krylov.pcg(A, b, precond=M, tol=1e-10, flexible=False)
    u1, i1 = krylov.pcg(A, b, precond=M, tol=1e-10, flexible=True)
    assert i0["converged"] and i1["converged"]
    assert abs(i0["iters"] - i1["iters"]) <= max(3, i0["iters"] // 10)
    # the same iterates up to rounding over the first iterations (rounding differences
    # then grow as the recurrences lose orthogonality)
    h0, h1 = np.array(i0["history"][:12]), np.array(i1["history"][:12])
    assert np.max(np.abs(h0 - h1) / h0) <= 1e-10
    np.testing.assert_allclose(u1, u0, rtol=0, atol=1e-8 * np.abs(u0).max())


def test_energy_norm_error_is_monotone():
    n = 50
    A = _spd(n, 78, cond=1e3)
    b = W.uniform01(79, n) - 0.5
    us = np.linalg.solve(A, b)
    errs = []
    for k in range(1, 25):
        u, _ = krylov.pcg(A, b, tol=0.0, maxit=k)
        e = u - us
        errs.append(float(e @ A @ e))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-10) for i in range(len(errs) - 1))


def test_restart_branch_replaces_the_recursive_residual():
    """Below the attainable accuracy the recursive residual keeps falling while
    the true one stalls: the solver replaces the residual by the true one and
    restarts, at most max_restarts times, then reports converged = False with
    the true relative residual of the returned iterate.  With an attainable
    tolerance the same system converges without a restart."""
    import scipy.sparse as sp
    n = 60
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat(np.logspace(0, 12, 6), n // 6)  # six clusters, condition 1e12
    A = sp.csr_matrix((Q * lam) @ Q.T)
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    u, info = krylov.pcg(A, b, tol=1e-12, maxit=2000, max_restarts=3)
    assert info["relres_recursive"] <= 1e-12  # the recursion met the tolerance ...
    assert info["restarts"] == 3 and not info["converged"], info["restarts"]
    true = np.linalg.norm(b - A @ u) / np.linalg.norm(b)
    assert abs(info["relres_true"] - true) <= 1e-12 * true
    assert info["relres_true"] > 1e-12  # ... the true residual did not
    u2, info2 = krylov.pcg(A, b, tol=1e-2, maxit=5000)
    assert info2["converged"] and info2["restarts"] == 0
