"""Whole-method parity: V-cycle (Algorithm 1) and preconditioned CG solves
through the C ABI vs the FP64 oracle (direct solve and the oracle's own MMG).

* FP64 form: solution within 1e-8 relative of the oracle's exact solution
  (solved to 1e-12), iteration count within +-2 of the oracle's MMG-PCG at
  1e-8 (bases agree to FP32-eigen accuracy, so the counts may differ by one
  or two at most).
* Mixed forms (FP32 V-cycle, BF16-storage smoother) inside FP64 flexible CG:
  the same 1e-8 solution accuracy once solved to 1e-12, error vs the oracle
  reported.
* Comparison modes (plain CG, Jacobi-PCG) reach the same solution.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from helpers import gpu_solver, oracle_problem, relerr, small_problem
from oracle import fem, krylov, mmg
import workloads as W

pytestmark = pytest.mark.gpu


def _exact(P):
    return spla.spsolve(P["A"].tocsc(), P["b"])


@pytest.fixture(scope="module")
def smooth32():
    pr = small_problem(32, kind="smooth")
    P = oracle_problem(pr)
    return pr, P, _exact(P)


def test_vcycle_fp64_matches_oracle(smooth32):
    pr, P, _ = smooth32
    s = gpu_solver(pr, prec=0)
    s.setup_precond()
    H = mmg.MMG(P)
    n = P["A"].shape[0]
    rng = np.random.default_rng(3)
    r = rng.standard_normal(n)
    r[P["mask"]] = 0.0
    z = s.vcycle(torch.as_tensor(r)).cpu().numpy()
    zo = H(r)
    assert relerr(z, zo) < 1e-4, relerr(z, zo)
    # symmetric and positive (FP64 V-cycle)
    y = rng.standard_normal(n)
    y[P["mask"]] = 0.0
    zy = s.vcycle(torch.as_tensor(y)).cpu().numpy()
    assert abs(z @ y - r @ zy) <= 1e-10 * np.linalg.norm(z) * np.linalg.norm(y)
    assert r @ z > 0
    s.close()


@pytest.mark.parametrize("case", [dict(N=64), dict(N=0, grid=(128, 64, 40), h=(1 / 128,) * 3)],
                         ids=["64", "box128x64x40"])
@pytest.mark.parametrize("prec,tol", [(1, 2e-5), (2, 5e-2)])
def test_vcycle_low_precision_matches_oracle(case, prec, tol):
    """The FP32 V-cycle (and the BF16-storage smoother variant) against the
    oracle's FP64 V-cycle (Algorithm 1 with the same Chebyshev smoother and
    hierarchy) on grids where the fine sweeps run two nodes per lane."""
    pr = small_problem(case["N"], kind="smooth", grid=case.get("grid"), h=case.get("h"))
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=prec)
    s.setup_precond()
    # the library's default hierarchy for these grids: 64^3 -> L (4, 8, 17); 128x64x40 -> (4, 17)
    opts = (mmg.default_options(case["N"]) if case["N"] else
            mmg.MMGOptions(block=4, nvec=(4, 17), group=(2,), smoother="chebyshev"))
    H = mmg.MMG(P, opts)
    assert [lv["nvec"] for lv in s.hierarchy()] == list(opts.nvec)
    n = P["A"].shape[0]
    r = np.random.default_rng(4).standard_normal(n)
    r[P["mask"]] = 0.0
    z = s.vcycle(torch.as_tensor(r)).cpu().numpy()
    assert relerr(z, H(r)) < tol, relerr(z, H(r))
    s.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_solve_matches_exact_solution(smooth32, prec):
    pr, P, ud = smooth32
    s = gpu_solver(pr, prec=prec)
    s.setup_precond()
    u, info = s.solve(tol=1e-12)
    u = u.cpu().numpy()
    assert info["rel_res_true"] <= 1e-12
    assert relerr(u, ud) < 1e-8, relerr(u, ud)
    s.close()


def test_fp64_iteration_count_matches_oracle(smooth32):
    pr, P, ud = smooth32
    H = mmg.MMG(P)
    _, io = krylov.pcg(P["A"], P["b"], precond=H, u0=H.coarse_guess(P["b"]), tol=1e-8)
    s = gpu_solver(pr, prec=0)
    s.setup_precond()
    u, info = s.solve(tol=1e-8)
    assert abs(info["iters"] - io["iters"]) <= 2, (info["iters"], io["iters"])
    assert info["rel_res_true"] <= 1e-8
    s.close()


@pytest.mark.parametrize("kind,N,kmin", [("chan", 32, 1e-6), ("thresh", 32, 1e-3), ("chan", 64, 1e-9)])
def test_high_contrast_solves(kind, N, kmin):
    pr = small_problem(N, kind=kind, seed=3, kmin=kmin)
    P = oracle_problem(pr)
    ud = _exact(P) if N <= 32 else None
    res = {}
    for prec in (0, 1, 2):
        s = gpu_solver(pr, prec=prec)
        s.setup_precond()
        u, info = s.solve(tol=1e-10)
        res[prec] = (u.cpu().numpy(), info)
        assert info["rel_res_true"] <= 1e-10, (prec, info)
        s.close()
    if ud is not None:
        for prec in (0, 1, 2):
            assert relerr(res[prec][0], ud) < 1e-6, (prec, relerr(res[prec][0], ud))
    else:
        # true FP64 residual of each solution, recomputed by the oracle
        for prec in (0, 1, 2):
            r = P["b"] - P["A"] @ res[prec][0]
            assert np.linalg.norm(r) <= 1.5e-10 * np.linalg.norm(P["b"])


@pytest.mark.parametrize("pc", [1, 2])
def test_comparison_modes(smooth32, pc):
    pr, P, ud = smooth32
    s = gpu_solver(pr, prec=0, pc=pc, guess=0, max_iter=20000)
    s.setup_precond()
    u, info = s.solve(tol=1e-11)
    assert relerr(u.cpu().numpy(), ud) < 1e-7
    _, io = krylov.pcg(P["A"], P["b"], precond=None if pc == 1 else krylov.jacobi_precond(P["A"]), tol=1e-11,
                       maxit=20000)
    assert abs(info["iters"] - io["iters"]) <= max(3, 0.02 * io["iters"]), (info["iters"], io["iters"])
    s.close()


def test_guess_modes_and_given_rhs(smooth32):
    pr, P, ud = smooth32
    s = gpu_solver(pr, prec=1, guess=2)
    s.setup_precond()
    u, info = s.solve(tol=1e-10)
    s2 = gpu_solver(pr, prec=1, guess=3)
    s2.setup_precond()
    u0 = torch.as_tensor(0.9 * ud)
    u2, info2 = s2.solve(u=u0.cuda(), tol=1e-10)
    assert relerr(u2.cpu().numpy(), ud) < 1e-7
    assert info2["iters"] <= info["iters"]
    rhs = torch.as_tensor(P["b"])
    u3, _ = s.solve(rhs=rhs, tol=1e-10)
    assert relerr(u3.cpu().numpy(), ud) < 1e-7
    s.close()
    s2.close()


def test_given_rhs_with_nonzero_dirichlet_entries(smooth32):
    """A caller's right-hand side is solved with the eliminated operator
    A = P_F A_N P_F + P_D (Sec. 2.1 boundary data): u_D = rhs_D exactly, the
    free part from A_FF u_F = rhs_F, whatever the Dirichlet values of the
    context were."""
    pr, P, ud = smooth32
    rhs = P["f"] + np.where(P["mask"], 0.5 + W.uniform01(5, P["f"].size), 0.0)
    ref = spla.spsolve(P["A"].tocsc(), rhs)
    for prec in (0, 1):
        s = gpu_solver(pr, prec=prec)
        s.setup_precond()
        u, info = s.solve(rhs=torch.as_tensor(rhs), tol=1e-11)
        u = u.cpu().numpy()
        assert np.array_equal(u[P["mask"]], rhs[P["mask"]])
        assert relerr(u, ref) < 1e-8, (prec, info)
        s.close()


def test_compliance_and_sensitivity_match_oracle(smooth32):
    pr, P, ud = smooth32
    s = gpu_solver(pr, prec=1)
    s.setup_precond()
    u, info = s.solve(tol=1e-12)
    c = s.compliance(u)
    co = fem.compliance(P["f"], ud)
    assert abs(c - co) <= 1e-10 * abs(co)
    dc = s.sensitivity(u).cpu().numpy()
    dco = fem.sensitivity(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], ud)
    assert relerr(dc, dco) < 1e-8
    s.close()


def test_nonzero_dirichlet_values_layered_exact():
    import workloads as W
    N = 16
    grid = (N, N, N)
    x = np.zeros((N, N, N))
    x[: N // 2] = 1.0
    vals = np.zeros((N + 1, N + 1, N + 1))
    vals[-1] = 1.0
    pr = dict(grid=grid, h=(1 / N,) * 3, mask=W.full_face_mask(grid, "z01"), source=np.zeros(N ** 3),
              x=x.ravel(), p=1.0, kmin=1e-6, kmax=1.0, values=vals.ravel())
    s = gpu_solver(pr, prec=1)
    s.setup_precond()
    u, info = s.solve(tol=1e-11)
    t = 1e-6 / (1 + 1e-6)
    z = np.arange(N + 1) / N
    prof = np.where(z <= 0.5, t * z / 0.5, t + (1 - t) * (z - 0.5) / 0.5)
    exact = (prof[:, None, None] * np.ones((1, N + 1, N + 1))).ravel()
    uu = u.cpu().numpy()
    np.testing.assert_allclose(uu, exact, atol=1e-9)
    lower = exact < 2 * t  # the conductive half carries values of order t = 1e-6
    np.testing.assert_allclose(uu[lower], exact[lower], rtol=1e-4, atol=1e-13)
    s.close()


def test_float_float_outer_operator_solve():
    """The mixed solve with the float-float outer operator (outer_apply = 2)
    at contrast 1e6 meets the tolerance on the oracle's assembled operator
    (true residual ||b - A u|| <= 1.5 tol ||b_F||, Dirichlet values exact),
    agrees with the FP64-arithmetic operator's solution to 1e-8, and takes
    its iteration count (+-2).  (A direct solve is too slow at 64^3.)"""
    pr = small_problem(64, kind="chan", kmin=1e-6)
    P = oracle_problem(pr)
    b, A, free = P["b"], P["A"], ~P["mask"]
    bF = np.linalg.norm(b[free])
    res, us = {}, {}
    for oa in (1, 2):
        s = gpu_solver(pr, prec=1, outer_apply=oa)
        s.setup_precond()
        u, info = s.solve(tol=1e-10)
        u = u.cpu().numpy()
        assert np.linalg.norm(b - A @ u) <= 1.5e-10 * bF, (oa, info)
        assert np.array_equal(u[P["mask"]], b[P["mask"]])
        res[oa], us[oa] = info["iters"], u
        s.close()
    assert relerr(us[2], us[1]) < 1e-8
    assert abs(res[2] - res[1]) <= 2, res


@pytest.mark.parametrize("prec,tol", [(0, 1e-4), (1, 2e-5)])
def test_wcycle_with_growing_sweeps_matches_oracle(prec, tol):
    """The cycle options of the deep levels (R17), active at 64^3 when the W-cycle
    starts at level 1: sweeps 1 / 2 on levels 1 / 2, two coarse corrections per
    level-1 visit; the GPU cycle (FP64 form, and FP32 with the two-nodes-per-lane
    engine) against the oracle's cycle with the same options."""
    pr = small_problem(64, kind="smooth")
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=prec, w_from=1, nu_growth=2)
    s.setup_precond()
    o = mmg.default_options(64)
    o.w_from, o.nu_growth = 1, 2
    H = mmg.MMG(P, o)
    n = P["A"].shape[0]
    r = np.random.default_rng(6).standard_normal(n)
    r[P["mask"]] = 0.0
    z = s.vcycle(torch.as_tensor(r)).cpu().numpy()
    assert relerr(z, H(r)) < tol, relerr(z, H(r))
    s.close()


@pytest.fixture(scope="module")
def uniform64():
    pr = small_problem(64, kind="rand", kmin=1e-3)
    pr["x"] = np.full(64 ** 3, 0.3)
    P = oracle_problem(pr)
    H = mmg.MMG(P)
    _, info = krylov.pcg(P["A"], P["b"], precond=H, u0=H.coarse_guess(P["b"]), tol=1e-8)
    return pr, P, info["iters"]


@pytest.mark.parametrize("prec", [0, 1])
def test_uniform_density_converges_like_the_oracle(uniform64, prec):
    """A uniform design (the first iterate of any SIMP loop): the Chebyshev
    interval must cover the dense top of the spectrum of D^-1 A.  Both forms
    converge, the FP64 form in the oracle's iteration count (+-2)."""
    pr, P, it_oracle = uniform64
    s = gpu_solver(pr, prec=prec)
    s.setup_precond()
    u, info = s.solve(tol=1e-8)
    assert info["iters"] <= 40, info
    if prec == 0:
        assert abs(info["iters"] - it_oracle) <= 2, (info["iters"], it_oracle)
    res = np.linalg.norm(P["b"] - P["A"] @ u.cpu().numpy()) / np.linalg.norm(P["b"][~P["mask"]])
    assert res <= 1.5e-8
    s.close()


@pytest.mark.parametrize("N", [32, 64])
def test_fp64_cycle_on_library_bases_matches_oracle(N):
    """One FP64 cycle (Algorithm 1: Chebyshev fine smoothing, fused residual +
    restriction, l1-block-Jacobi coarse levels with the W-cycle below level 3,
    direct coarsest solve, prolongations) against the oracle's cycle built on
    the library's own exported bases, so that the comparison isolates the
    cycle's arithmetic from the two eigensolvers.  Smooth design (kmin 1e-3):
    the coarsest operator is well conditioned, so the explicit inverse and the
    oracle's Cholesky solve agree to about 1e-14."""
    from helpers import library_bases
    pr = small_problem(N, kind="smooth")
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=0)
    s.setup_precond()
    G = mmg.MMG(P, mmg.default_options(N), bases=library_bases(s, pr))
    n = P["A"].shape[0]
    rng = np.random.default_rng(N)
    for _ in range(2):
        r = rng.standard_normal(n)
        r[P["mask"]] = 0.0
        z = s.vcycle(torch.as_tensor(r)).cpu().numpy()
        assert relerr(z, G(r)) < 1e-11, relerr(z, G(r))
    s.close()


@pytest.mark.parametrize("kind,kmin", [("smooth", 1e-3), ("chan", 1e-6)])
def test_coarse_guess_is_the_galerkin_solution(kind, kmin):
    """The interpolated coarse initial guess u0 = P A_L^-1 P^T b: taken from a
    solve whose tolerance the guess already meets (the CG loop does not run),
    it satisfies Galerkin orthogonality P^T (b - A u0) = 0 for the library's
    composite prolongation P (rebuilt from its exported bases), and equals the
    oracle's coarse guess on those bases; on a smooth design (simple local
    spectra) it also agrees with the oracle's guess on the oracle's own bases.
    (At high contrast, near-degenerate local eigenvalues at the cut-off let the
    two eigensolvers pick different but equally valid coarse spaces.)"""
    from helpers import library_bases
    pr = small_problem(32, kind=kind, seed=3, kmin=kmin)
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=0)
    s.setup_precond()
    u0, info = s.solve(tol=1e300)
    assert info["iters"] == 0
    u0 = u0.cpu().numpy()
    bases = library_bases(s, pr)
    Pc = bases[0]
    for B in bases[1:]:
        Pc = Pc @ B
    res = Pc.T @ (P["b"] - P["A"] @ u0)
    assert np.linalg.norm(res) <= 1e-12 * np.linalg.norm(Pc.T @ P["b"]), np.linalg.norm(res)
    G = mmg.MMG(P, mmg.default_options(32), bases=bases)
    assert relerr(u0, G.coarse_guess(P["b"])) < 1e-12
    if kind == "smooth":
        # simple local spectra: the two eigensolvers give the same coarse spaces
        H = mmg.MMG(P)
        assert relerr(u0, H.coarse_guess(P["b"])) < 1e-4
    s.close()


def test_fp32_density_input_matches_fp64_input():
    """opt.density_fp32: thermo_set_density reads float x (widened on the
    device); for an FP32-representable design the solution is bitwise the one
    of the FP64 input."""
    pr = small_problem(32, kind="smooth")
    x32 = pr["x"].astype(np.float32)
    s64 = gpu_solver(dict(pr, x=x32.astype(np.float64)), prec=1)
    s32 = gpu_solver(dict(pr, x=x32), prec=1, density_fp32=1)
    out = []
    for s in (s64, s32):
        s.setup_precond()
        u, info = s.solve(tol=1e-10)
        out.append((u.cpu().numpy(), info["iters"], s.sensitivity(u).cpu().numpy()))
        s.close()
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][2], out[1][2])


def test_update_density_keeps_the_preconditioner():
    """thermo_update_density: a perturbed design is solved with the preconditioner
    of the earlier design (no new set-up), to the oracle's residual on the new
    operator; thermo_set_density instead marks the preconditioner stale."""
    pr = small_problem(32, kind="smooth", kmin=1e-3)
    s = gpu_solver(pr, prec=1)
    s.setup_precond()
    u0, i0 = s.solve(tol=1e-10)
    x2 = pr["x"].copy()
    for e in (100, 5000, 20000):  # finite-difference sized perturbations
        x2[e] += 1e-3
    s.update_density(torch.as_tensor(x2), pr["p"], pr["kmin"], pr["kmax"])
    u, info = s.solve(tol=1e-10)
    P = oracle_problem(dict(pr, x=x2))
    res = P["b"] - P["A"] @ u.cpu().numpy()
    assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(P["b"])
    assert info["iters"] <= i0["iters"] + 2, (info["iters"], i0["iters"])
    from paper_2410_06850_gb300 import ThermoError, thermo
    s.set_density(torch.as_tensor(x2), pr["p"], pr["kmin"], pr["kmax"])
    with pytest.raises(ThermoError) as e:
        s.solve()
    assert e.value.status == thermo.ESTATE
    s.close()


@pytest.mark.parametrize("grid", [(40, 44, 36), (40, 40, 40)])
def test_mixed_solve_on_partial_tiles(grid):
    """Mixed-form solves whose FP32 sweeps run on partial tiles of the separable
    engine in x, y and z, to the oracle's true residual and its exact solution."""
    pr = small_problem(0, kind="rand", kmin=1e-3, grid=grid, h=(1.0 / grid[1],) * 3)
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=1)
    s.setup_precond()
    u, info = s.solve(tol=1e-11)
    u = u.cpu().numpy()
    assert np.linalg.norm(P["b"] - P["A"] @ u) <= 1.5e-11 * np.linalg.norm(P["b"])
    assert relerr(u, _exact(P)) < 1e-8
    s.close()
