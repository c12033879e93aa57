"""Conjugate-gradient solvers (oracle, test infrastructure only).

The paper solves both linear systems with PETSc CG wrapped around the MMG
preconditioner (Sec. 4, experimental setup).  The stopping rule used here is
the unpreconditioned 2-norm relative to the free part of the right-hand side:
||b - A u_k|| <= tol ||b_F|| (Dirichlet rows are identities and carry no
residual once u holds the boundary values),
checked on the recursive residual and confirmed on the true residual at exit
(on failure of the confirmation the residual is replaced by the true one and
the iteration restarts from the current iterate).

Iteration count = number of products A p inside the loop, which equals the
number of preconditioner applications (the initial one included).

``flexible=True`` uses the Polak-Ribiere coefficient
beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k, which stays a descent method for a
preconditioner that varies between applications (e.g. one evaluated in lower
precision).
"""
from __future__ import annotations

import numpy as np


def pcg(A, b, precond=None, u0=None, tol=1e-8, maxit=10000, flexible=False,
        max_restarts=5, free=None):
    """Returns (u, info) with info = dict(iters, converged, relres_recursive,
    relres_true, history).  ``free``: boolean mask of the unknowns that are
    not Dirichlet rows; the relative residual is measured against ||b_F||
    (the identity rows hold exactly for every iterate that starts with the
    Dirichlet values)."""
    n = b.shape[0]
    u = np.zeros(n) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
    M = (lambda r: r.copy()) if precond is None else precond
    bnorm = float(np.linalg.norm(b if free is None else b[free]))
    if bnorm == 0.0:
        return np.zeros(n), dict(iters=0, converged=True, relres_recursive=0.0,
                                 relres_true=0.0, history=[0.0])
    r = b - A @ u
    hist = [float(np.linalg.norm(r)) / bnorm]
    it = 0
    restarts = 0
    if hist[-1] <= tol:
        return u, dict(iters=0, converged=True, relres_recursive=hist[-1],
                       relres_true=hist[-1], history=hist)
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    converged = False
    while it < maxit:
        q = A @ p
        pq = float(p @ q)
        if not np.isfinite(pq) or pq <= 0.0:
            break
        alpha = rz / pq
        u += alpha * p
        r -= alpha * q
        it += 1
        rz_old_new_r = float(r @ z)  # r_{k+1} . z_k (flexible numerator term)
        rnorm = float(np.linalg.norm(r))
        hist.append(rnorm / bnorm)
        if rnorm <= tol * bnorm:
            rt = b - A @ u
            if float(np.linalg.norm(rt)) <= tol * bnorm or restarts >= max_restarts:
                converged = float(np.linalg.norm(rt)) <= tol * bnorm
                break
            restarts += 1
            r = rt
            z = M(r)
            p = z.copy()
            rz = float(r @ z)
            continue
        z = M(r)
        rz_new = float(r @ z)
        beta = (rz_new - rz_old_new_r) / rz if flexible else rz_new / rz
        rz = rz_new
        p = z + beta * p
    rt = b - A @ u
    return u, dict(iters=it, converged=converged, restarts=restarts,
                   relres_recursive=hist[-1],
                   relres_true=float(np.linalg.norm(rt)) / bnorm, history=hist)


def jacobi_precond(A):
    """Point-Jacobi preconditioner z = D^-1 r (comparison mode)."""
    d = A.diagonal().copy()
    inv = 1.0 / d
    return lambda r: inv * r
