"""SIMP harness and differentiation on the GPU:
* density filter and its transpose vs the oracle's sparse filter matrix;
* one OC update vs the oracle's bisection on the same inputs;
* ComplianceFn (torch.autograd) gradient vs the oracle's adjoint formula and
  vs central finite differences of the compliance on a small grid;
* the adjoint sensitivity within 1e-6 of central differences formed without
  cancellation (one extra solve per perturbed design)."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import gpu_solver, oracle_problem, relerr, small_problem
from oracle import fem, topopt
from paper_2410_06850_gb300 import autograd as AG

pytestmark = pytest.mark.gpu


def test_filter_and_transpose_match_oracle():
    N = 16
    pr = small_problem(N)
    s = gpu_solver(pr)
    H = topopt.filter_matrix(N, 1.5)
    x = W.uniform01(3, N ** 3)
    y = s.filter(torch.as_tensor(x), 1.5).cpu().numpy()
    np.testing.assert_allclose(y, H @ x, rtol=1e-13)
    yt = s.filter(torch.as_tensor(x), 1.5, transpose=True).cpu().numpy()
    np.testing.assert_allclose(yt, H.T @ x, rtol=1e-13)
    s.close()


def test_oc_update_matches_oracle():
    N = 16
    pr = small_problem(N)
    s = gpu_solver(pr)
    H = topopt.filter_matrix(N, 1.5)
    x = 0.2 + 0.2 * W.uniform01(4, N ** 3)
    dc = -(0.1 + W.uniform01(5, N ** 3))
    dv = np.ones(N ** 3)
    xo = topopt.oc_update(x, dc, dv, 0.3, H=H, move=0.2)
    xt = torch.as_tensor(x).cuda()
    s.oc_update(xt, torch.as_tensor(dc).cuda(), torch.as_tensor(dv).cuda(), 0.3, 0.2, 1.5)
    np.testing.assert_allclose(xt.cpu().numpy(), xo, rtol=1e-9, atol=1e-12)
    assert abs((H @ xo).mean() - 0.3) < 2e-3
    s.close()


def test_compliance_autograd_matches_adjoint_and_fd():
    N = 16
    pr = small_problem(N, kind="smooth", kmin=1e-2)
    s = gpu_solver(pr, prec=0)
    x = torch.as_tensor(pr["x"]).cuda().requires_grad_(True)
    c = AG.compliance(x, s, pr["p"], pr["kmin"], pr["kmax"], tol=1e-12)
    c.backward()
    g = x.grad.cpu().numpy()
    P = oracle_problem(pr)
    import scipy.sparse.linalg as spla
    ud = spla.spsolve(P["A"].tocsc(), P["b"])
    go = fem.sensitivity(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], ud)
    assert relerr(g, go) < 1e-9
    assert abs(c.item() - fem.compliance(P["f"], ud)) <= 1e-12 * abs(c.item())
    # central differences of the GPU compliance on a few elements
    for e in [0, 1000, 2047, 4095]:
        d = 1e-4
        cs = []
        for sg in (+1, -1):
            xp = x.detach().clone()
            xp[e] += sg * d
            cs.append(AG.compliance(xp, s, pr["p"], pr["kmin"], pr["kmax"], tol=1e-12).item())
        fd = (cs[0] - cs[1]) / (2 * d)
        assert abs(fd - g[e]) <= 1e-4 * abs(g[e]) + 1e-9 * abs(c.item()), (e, fd, g[e])
    s.close()


def test_filter_autograd_is_transpose():
    N = 8
    pr = small_problem(N)
    s = gpu_solver(pr)
    x = torch.as_tensor(W.uniform01(8, N ** 3)).cuda().requires_grad_(True)
    w = torch.as_tensor(W.uniform01(9, N ** 3)).cuda()
    y = AG.density_filter(x, s, 1.5)
    (y * w).sum().backward()
    H = topopt.filter_matrix(N, 1.5)
    np.testing.assert_allclose(x.grad.cpu().numpy(), H.T @ w.cpu().numpy(), rtol=1e-12)
    s.close()


def _interior_elements(x, count, seed, margin):
    cand = (W.uniform01(seed, 4 * count) * x.size).astype(np.int64)
    cand = [int(e) for e in cand if margin <= x[e] <= 1.0 - margin]
    return list(dict.fromkeys(cand))[:count]


def test_sensitivity_within_1e6_of_exact_central_differences():
    """dc/dx_e of the adjoint kernel (Sec. 2.3) against central differences of
    the compliance c = f^T u, formed without cancellation.  For x' = x + s d e_e,
    with dK = (kappa'_e - kappa_e) K0 on the element's free nodes and A' the
    perturbed operator, c' - c = -u_e^T dK u_e + w_e^T dK u_e with A' w = dK u
    (A' symmetric, T = 0 on Gamma_D).  That is one extra solve per perturbed
    design; its term is second order in d, so its rounding hardly matters.  The
    central quotient's truncation error is O(d^2), about 1e-8 at d = 1e-4.  All
    solves are in the FP64 form to 1e-12."""
    N = 16
    pr = small_problem(N, kind="smooth", kmin=1e-2)
    grid, h = pr["grid"], pr["h"]
    p, kmin, kmax = pr["p"], pr["kmin"], pr["kmax"]
    s = gpu_solver(pr, prec=0)
    s.setup_precond()
    u, _ = s.solve(tol=1e-12)
    g = s.sensitivity(u).cpu().numpy()
    u = u.cpu().numpy()
    K0 = fem.element_matrix(h)
    en = fem.element_nodes(grid)
    free = ~pr["mask"].astype(bool)
    n = fem.n_nodes(grid)
    d = 1e-4
    elems = _interior_elements(pr["x"], 6, 61, 4 * d)
    assert len(elems) >= 4
    for e in elems:
        nodes = en[e]
        fe = free[nodes].astype(np.float64)
        ue = u[nodes] * fe
        k0 = fem.simp_kappa(pr["x"][e], p, kmin, kmax)
        dc = []
        for sg in (+1.0, -1.0):
            xp = pr["x"].copy()
            xp[e] += sg * d
            dk = fem.simp_kappa(xp[e], p, kmin, kmax) - k0
            dKu = dk * (K0 @ ue) * fe
            rhs = np.zeros(n)
            rhs[nodes] = dKu
            s.set_density(torch.as_tensor(xp), p, kmin, kmax)
            s.setup_precond()
            w, _ = s.solve(rhs=torch.as_tensor(rhs), tol=1e-12)
            we = w.cpu().numpy()[nodes] * fe
            dc.append(-(ue @ dKu) + we @ dKu)
        fd = (dc[0] - dc[1]) / (2.0 * d)
        assert abs(fd - g[e]) <= 1e-6 * abs(g[e]), (e, fd, g[e])
    s.close()
