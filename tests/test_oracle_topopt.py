"""Pins of the oracle's SIMP harness (density filter and OC update; textbook
SIMP that drives the repeated solves of Sec. 2.3, not the paper's MMA):

* the filter against a brute-force loop over all element pairs on tiny grids,
  its row sums, the identity at radius <= 1 and its transpose;
* the OC step's box and move limits, the volume it reaches, its closed form on
  uniform sensitivities, and the optimality form x_new = x (-dc / (lambda dv))^eta
  shared by every element that no limit clips.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import topopt


def brute_filter(N, rmin):
    """Hat weights max(0, rmin - |c_e - c_j|) between element centroids, summed
    over the elements of the grid only, each row divided by its sum."""
    M = N ** 3
    H = np.zeros((M, M))
    for e in range(M):
        ex, ey, ez = e % N, (e // N) % N, e // (N * N)
        for j in range(M):
            jx, jy, jz = j % N, (j // N) % N, j // (N * N)
            d = np.sqrt((ex - jx) ** 2 + (ey - jy) ** 2 + (ez - jz) ** 2)
            H[e, j] = max(0.0, rmin - d)
        H[e] /= H[e].sum()
    return H


@pytest.mark.parametrize("N,rmin", [(3, 1.5), (4, 2.0), (4, 2.5), (5, 1.2)])
def test_filter_matches_brute_force(N, rmin):
    H = topopt.filter_matrix(N, rmin).toarray()
    np.testing.assert_allclose(H, brute_filter(N, rmin), rtol=0, atol=1e-15)


@pytest.mark.parametrize("rmin", [0.5, 1.0])
def test_filter_radius_at_most_one_is_identity(rmin):
    H = topopt.filter_matrix(4, rmin)
    assert abs(H - sp.identity(64)).max() == 0.0


def test_filter_rows_sum_to_one_and_transpose():
    N = 6
    H = topopt.filter_matrix(N, 1.5)
    np.testing.assert_allclose(np.asarray(H.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-15)
    x = W.uniform01(31, N ** 3)
    y = W.uniform01(32, N ** 3)
    np.testing.assert_allclose(H @ np.full(N ** 3, 0.37), 0.37, rtol=0, atol=1e-15)
    assert abs((H @ x) @ y - x @ (H.T @ y)) <= 1e-13 * abs(x @ (H.T @ y))
    # the filter is not symmetric at the boundary (rows are normalised), so H^T != H
    assert abs(H - H.T).max() > 1e-3


def test_oc_uniform_sensitivities_give_the_target_volume():
    # closed form: with dc and dv uniform every element gets x (1 / (lambda dv))^eta,
    # a uniform design; the bisection puts it at the target within its tolerance
    M = 200
    x = np.full(M, 0.5)
    xn = topopt.oc_update(x, -np.ones(M), np.ones(M), 0.4)
    assert np.ptp(xn) == 0.0
    assert abs(xn[0] - 0.4) <= 1e-3


def test_oc_move_limit_binds():
    M = 50
    x = np.full(M, 0.5)
    xn = topopt.oc_update(x, -np.ones(M), np.ones(M), 0.1, move=0.2)
    np.testing.assert_array_equal(xn, 0.3)  # x - move: the target volume is out of reach


def test_oc_limits_volume_and_optimality_form():
    N = 6
    M = N ** 3
    H = topopt.filter_matrix(N, 1.5)
    x = 0.2 + 0.6 * W.uniform01(33, M)
    dc = -(0.01 + W.uniform01(34, M) ** 3)
    dv = np.ones(M)
    move, eta, vf = 0.2, 0.5, 0.35
    xn = topopt.oc_update(x, dc, dv, vf, H=H, move=move, eta=eta)
    lo, hi = np.maximum(0.0, x - move), np.minimum(1.0, x + move)
    assert np.all(xn >= lo) and np.all(xn <= hi)
    assert abs((H @ xn).mean() - vf) <= 5e-3
    free = (xn > lo + 1e-12) & (xn < hi - 1e-12)
    assert free.sum() > M // 4
    # on the unclipped elements (xn / x)^(1/eta) * dv / (-dc) = 1 / lambda, one value for all
    inv_lam = (xn[free] / x[free]) ** (1.0 / eta) * dv[free] / (-dc[free])
    assert np.ptp(inv_lam) <= 1e-12 * inv_lam.mean()
    # and the ordering of -dc / x^... : a larger -dc never gives a smaller step ratio
    order = np.argsort(-dc[free])
    assert np.all(np.diff((xn[free] / x[free])[order]) >= -1e-15)
