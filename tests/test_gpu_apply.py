"""Fine operator apply through the C ABI vs the oracle's assembled CSR matrix
(Sec. 2.2 Eq. (5) realised with Q1 elements), element by element.

Sizes span one and several x/y/z tiles and the ragged closing node plane;
one case uses non-cubic elements (27-point stencil) and a non-cubic grid;
inputs are nonzero on Dirichlet nodes to exercise the identity rows.
"""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import gpu_solver, oracle_problem, small_problem

pytestmark = pytest.mark.gpu

CASES = [
    dict(N=8),
    dict(N=16),
    dict(N=32),
    dict(N=64),
    dict(N=16, grid=(16, 8, 12), h=(0.05, 0.07, 0.04)),
    dict(N=32, grid=(32, 64, 16)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: str(c.get("grid", c["N"])))
def test_apply_fp64_matches_oracle(case):
    pr = small_problem(case["N"], grid=case.get("grid"), h=case.get("h"), kind="rand", kmin=1e-6)
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=0)
    n = P["A"].shape[0]
    u = W.uniform01(5, n) - 0.3
    y = s.apply(torch.as_tensor(u), 0).cpu().numpy()
    ref = P["A"] @ u
    scale = np.abs(P["A"]).dot(np.abs(u))
    err = np.abs(y - ref) / np.maximum(scale, 1e-300)
    assert err.max() < 1e-13, err.max()
    s.close()


LP_CASES = [dict(N=32), dict(N=64), dict(N=0, grid=(128, 64, 40), h=(1 / 128,) * 3),
            dict(N=0, grid=(40, 44, 36), h=(1 / 44,) * 3), dict(N=96),
            dict(N=64, engine=1), dict(N=0, grid=(32, 16, 24), h=(1 / 32, 1 / 16, 1 / 24))]


@pytest.mark.parametrize("case", LP_CASES, ids=["32", "64", "box128x64x40", "box40x44x36", "96",
                                                 "64_two_per_lane", "box32x16x24_noncubic"])
@pytest.mark.parametrize("prec,tol", [(1, 2e-6), (2, 3e-2)])
def test_apply_low_precision_normwise(prec, tol, case):
    """FP32 and BF16-storage applies.  FP32 on cubic elements: the separable
    engine (tiles of 30 x 32 nodes, so these grids end in partial tiles in x and
    y, and 97 nodes leave a one-row last tile); engine 1 and BF16 storage: two
    nodes per lane (Nx a multiple of 64) or one node per lane; non-cubic
    elements: one node per lane."""
    pr = small_problem(case["N"], kind="rand", kmin=1e-3, grid=case.get("grid"), h=case.get("h"))
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=prec, fine_engine=case.get("engine", 0))
    n = P["A"].shape[0]
    u = W.uniform01(6, n) - 0.5
    y = s.apply(torch.as_tensor(u), prec).cpu().numpy()
    ref = P["A"] @ u
    scale = np.abs(P["A"]).dot(np.abs(u))
    err = np.abs(y - ref) / np.maximum(scale, 1e-300)
    assert err.max() < tol, err.max()
    assert np.array_equal(y[P["mask"]], u[P["mask"]])  # identity rows
    s.close()


def test_load_vector_matches_oracle():
    pr = small_problem(16)
    pr["source"] = 1.0 + W.uniform01(9, 16 ** 3)
    P = oracle_problem(pr)
    s = gpu_solver(pr)
    f = s.load_vector().cpu().numpy()
    np.testing.assert_allclose(f, P["f"], rtol=1e-14, atol=0)
    s.close()


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_fused_apply_dot_matches(N):
    """The fused q = A p, p.Ap kernel of the CG loop equals the plain apply and
    the dot product (p zero on Gamma_D, as for CG directions)."""
    pr = small_problem(N, kind="rand", kmin=1e-4)
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=0)
    n = P["A"].shape[0]
    p = W.uniform01(11, n) - 0.4
    p[P["mask"]] = 0.0
    q, pq = s.apply_dot(torch.as_tensor(p))
    q = q.cpu().numpy()
    ref = P["A"] @ p
    scale = np.abs(P["A"]).dot(np.abs(p))
    assert (np.abs(q - ref) / np.maximum(scale, 1e-300)).max() < 1e-13
    assert abs(pq - p @ ref) <= 1e-12 * abs(p @ ref)
    s.close()


# The float-float (FP64-accurate, FP32-pipe) outer operator: cubic elements and
# Nx a multiple of 64.  Cases: a cube (one x tile: closing column in every CTA
# row), and a box of cube elements with two x tiles and a ragged z chunk.
FF_CASES = [dict(N=64), dict(N=0, grid=(128, 64, 40), h=(1 / 128,) * 3)]


@pytest.mark.parametrize("case", FF_CASES, ids=["cube64", "box128x64x40"])
@pytest.mark.parametrize("smooth_p", [False, True], ids=["random_p", "smooth_p"])
def test_float_float_apply_dot_matches_oracle(case, smooth_p):
    """Sec. 2.2 Eq. (5) in difference form with float-float arithmetic: q within
    1e-13 of the oracle's assembled A p relative to |A||p| row by row, p.q
    within 1e-12, on random and on smooth directions (the cancelling case),
    and equal to the FP64-arithmetic kernel to the same bound."""
    pr = small_problem(case["N"], kind="rand", kmin=1e-6, grid=case.get("grid"), h=case.get("h"))
    P = oracle_problem(pr)
    n = P["A"].shape[0]
    if smooth_p:
        gx, gy, gz = (np.arange(k + 1) / k for k in pr["grid"])
        p = (np.sin(2.1 * gz)[:, None, None] * np.cos(1.3 * gy)[None, :, None] *
             (1.0 + gx)[None, None, :]).ravel() * 1e3
    else:
        p = W.uniform01(13, n) - 0.4
    p[P["mask"]] = 0.0
    ref = P["A"] @ p
    scale = np.abs(P["A"]).dot(np.abs(p))
    qs = {}
    for oa in (2, 1):
        s = gpu_solver(pr, prec=1, outer_apply=oa)
        q, pq = s.apply_dot(torch.as_tensor(p))
        q = q.cpu().numpy()
        assert (np.abs(q - ref) / np.maximum(scale, 1e-300)).max() < 1e-13, oa
        assert abs(pq - p @ ref) <= 1e-12 * abs(p @ ref), oa
        qs[oa] = q
        s.close()
    assert (np.abs(qs[2] - qs[1]) / np.maximum(scale, 1e-300)).max() < 1e-13
