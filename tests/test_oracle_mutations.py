"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in
the oracle on the CPU (a dropped term, a wrong sign, a wrong exponent or index,
a missing normalisation or elimination), re-runs the pins that guard that
function, and requires that at least one of them fails.  The oracle itself is
restored after each case (pytest monkeypatch).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import test_oracle_fem as F
import test_oracle_mmg as G
import test_oracle_resample as R
import test_oracle_topopt as T
import test_oracle_tpfa as TP
from oracle import fem, mmg, topopt, tpfa

_K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
_M1 = np.array([[1.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 1.0 / 3.0]])
_orig = {"element_matrix": fem.element_matrix, "simp_kappa": fem.simp_kappa, "load_vector": fem.load_vector,
         "sensitivity": fem.sensitivity, "filter_matrix": topopt.filter_matrix,
         "sensitivity_at": fem.sensitivity_at, "load_rows": fem.load_rows,
         "cells": topopt._axis_weights_cells, "kept_count": mmg.kept_count,
         "tpfa_assemble": tpfa.assemble, "tpfa_sensitivity": tpfa.sensitivity}


def k_dropped_term(h):
    hx, hy, hz = (float(v) for v in h)
    return (hy * hz / hx) * np.kron(_M1, np.kron(_M1, _K1)) + (hx * hz / hy) * np.kron(_M1, np.kron(_K1, _M1))


def k_axes_swapped(h):
    # the x and z factors exchanged (local index read as az + 2ay + 4ax)
    hx, hy, hz = (float(v) for v in h)
    K = (hy * hz / hx) * np.kron(_K1, np.kron(_M1, _M1))
    K += (hx * hz / hy) * np.kron(_M1, np.kron(_K1, _M1))
    K += (hx * hy / hz) * np.kron(_M1, np.kron(_M1, _K1))
    return K


def kappa_wrong_exponent(x, p, kmin, kmax):
    return _orig["simp_kappa"](x, p - 1.0, kmin, kmax)


def load_double_weight(grid, h, source):
    return 2.0 * _orig["load_vector"](grid, h, source)


def sensitivity_wrong_sign(grid, h, x, p, kmin, kmax, u):
    return -_orig["sensitivity"](grid, h, x, p, kmin, kmax, u)


def sensitivity_wrong_power(grid, h, x, p, kmin, kmax, u):
    x = np.asarray(x, float)
    return -p * x ** p * (kmax - kmin) * fem.element_energy(grid, h, u)


def dirichlet_rows_only(A_neu, f, mask, values=None):
    # identity rows on Gamma_D but the Dirichlet columns kept in the free rows
    mask = np.asarray(mask).astype(bool)
    free = (~mask).astype(np.float64)
    A = (sp.diags(free) @ A_neu + sp.diags(mask.astype(np.float64))).tocsr()
    return A, free * f


def filter_unnormalised(N, rmin):
    H = _orig["filter_matrix"](N, rmin)
    H = H.tocoo()
    # rows scaled by their neighbour counts: they no longer sum to one
    w = np.zeros(N ** 3)
    np.add.at(w, H.row, H.data > 0)
    return sp.csr_matrix((H.data * w[H.row], (H.row, H.col)), shape=H.shape)


def l1_without_abs(A, shape, L):
    A = A.tocsr()
    ncell = shape[0] * shape[1] * shape[2]
    rows = np.asarray(A.sum(axis=1)).ravel()
    out = []
    for c in range(ncell):
        d = np.arange(c * L, (c + 1) * L)
        D = A[d][:, d].toarray()
        inside = np.asarray(A[d][:, d].sum(axis=1)).ravel()
        out.append(np.linalg.inv(D + np.diag(rows[d] - inside)))
    return out


def cell_weights_swapped(N, r):
    i0, i1, t = _orig["cells"](N, r)
    return i0, i1, np.where(i0 == i1, t, 1.0 - t)  # the weight of the nearer centre on the farther one


def node_weights_no_closing_node(N, r):
    i = np.arange(N * r + 1)
    i0 = np.minimum(i // r, N - 1)
    return i0, i0 + 1, (i % r) / r  # the last node (i = rN) read as the start of cell N-1


def kept_one_more(w, L, thr):
    k = _orig["kept_count"](w, L, thr)
    return min(k + 1, min(L, len(w))) if thr > 0 else k


def sensitivity_at_wrong_power(grid, h, x_e, p, kmin, kmax, u, elems):
    x = np.asarray(x_e, float)
    return _orig["sensitivity_at"](grid, h, x, p, kmin, kmax, u, elems) * x  # x^p in place of x^(p-1)


def load_rows_without_eighth(grid, h, source, rows):
    return 8.0 * _orig["load_rows"](grid, h, source, rows)


def tpfa_full_cell_dirichlet(grid, h, kappa, dfaces):
    # the Dirichlet face's distance taken as a whole cell instead of half of one
    A, tauD = _orig["tpfa_assemble"](grid, h, kappa, dfaces)
    half = {k: 0.5 * v for k, v in tauD.items()}
    corr = sum(half.values())
    return (A - sp.diags(corr)).tocsr(), half


def tpfa_sensitivity_no_source(P, t, u):
    Q = dict(P, source_given=True)  # drops the -f0 p x^(p-1) |K| u term
    return _orig["tpfa_sensitivity"](Q, t, u)


CASES = {
    "element matrix drops a term": (fem, "element_matrix", k_dropped_term,
                                    [lambda: F.test_element_matrix_matches_gauss_quadrature((0.3, 0.5, 0.7)),
                                     F.test_element_matrix_cube_closed_form]),
    "element matrix axes swapped": (fem, "element_matrix", k_axes_swapped,
                                    [lambda: F.test_element_matrix_matches_gauss_quadrature((0.3, 0.5, 0.7))]),
    "SIMP exponent p - 1": (fem, "simp_kappa", kappa_wrong_exponent,
                            [F.test_sensitivity_euler_identity, F.test_sensitivity_central_finite_differences]),
    "load vector weight": (fem, "load_vector", load_double_weight,
                           [F.test_load_vector_integrates_source, F.test_compliance_energy_identity_and_mean_temperature]),
    "sensitivity sign": (fem, "sensitivity", sensitivity_wrong_sign,
                         [F.test_sensitivity_euler_identity, F.test_sensitivity_central_finite_differences]),
    "sensitivity power p": (fem, "sensitivity", sensitivity_wrong_power,
                            [F.test_sensitivity_euler_identity, F.test_sensitivity_central_finite_differences]),
    "Dirichlet columns kept": (fem, "dirichlet_system", dirichlet_rows_only,
                               [F.test_operator_symmetric_spd_zero_rowsums_mmatrix]),
    "filter rows not normalised": (topopt, "filter_matrix", filter_unnormalised,
                                   [lambda: T.test_filter_matches_brute_force(3, 1.5),
                                    T.test_filter_rows_sum_to_one_and_transpose]),
    "l1 smoother without |a_ij|": (mmg, "l1_block_inverses", l1_without_abs,
                                   [G.test_l1_block_jacobi_is_convergent_without_damping]),
    "resample: cell weights swapped": (topopt, "_axis_weights_cells", cell_weights_swapped,
                                       [lambda: R.test_cell_trilinear_pointwise((3, 2, 4), (6, 4, 8)),
                                        R.test_cell_trilinear_reproduces_linear_fields_inside]),
    "resample: closing node misplaced": (topopt, "_axis_weights_nodes", node_weights_no_closing_node,
                                         [lambda: R.test_nodal_embedding_pointwise((3, 2, 4), (6, 4, 8)),
                                          lambda: R.test_nodal_embedding_keeps_integral_and_energy((3, 2, 4),
                                                                                                   (6, 4, 8))]),
    "adaptive count one too many": (mmg, "kept_count", kept_one_more,
                                    [G.test_adaptive_count_equals_high_conductivity_components]),
    "listed-element sensitivity power p": (fem, "sensitivity_at", sensitivity_at_wrong_power,
                                           [lambda: F.test_sampled_load_and_sensitivity_equal_the_full_ones(
                                               (6, 4, 5), (0.3, 0.5, 0.7))]),
    "listed-node load without 1/8": (fem, "load_rows", load_rows_without_eighth,
                                     [lambda: F.test_sampled_load_and_sensitivity_equal_the_full_ones(
                                         (6, 4, 5), (0.3, 0.5, 0.7))]),
    "TPFA: full-cell Dirichlet distance": (tpfa, "assemble", tpfa_full_cell_dirichlet,
                                           [lambda: TP.test_series_conduction_is_exact(8)]),
    "TPFA: sensitivity without the source term": (tpfa, "sensitivity", tpfa_sensitivity_no_source,
                                                  [lambda: TP.test_adjoint_identity_and_central_differences(
                                                      "z0_full", 0.0)]),
}


@pytest.mark.parametrize("name", list(CASES))
def test_pins_catch_a_planted_mistake(monkeypatch, name):
    mod, attr, bad, pins = CASES[name]
    monkeypatch.setattr(mod, attr, bad)
    caught = 0
    for pin in pins:
        try:
            pin()
        except (AssertionError, np.linalg.LinAlgError):
            caught += 1
    assert caught >= 1, f"no pin caught: {name}"


def test_tpfa_arithmetic_face_mean_is_caught():
    """The arithmetic instead of the harmonic face mean (computed here directly,
    not by patching) breaks the 1-D series-conduction exactness."""
    grid = (1, 1, 6)
    kz = np.array([1e-3, 1.0, 1e-2, 1.0, 1e-1, 1.0])
    dfaces = tpfa.dirichlet_faces(grid, "z0z1_full")
    P = tpfa.build(grid, (1.0, 1.0, 1 / 6), kz, 1.0, 0.0, 1.0, 0.0, dfaces, TD={(2, 0): 0.0, (2, 1): 1.0})
    A = P["A"].toarray()
    h = 1 / 6
    for k in range(5):  # replace every harmonic face transmissibility by the arithmetic one
        harm = -A[k, k + 1]
        arith = 0.5 * (kz[k] + kz[k + 1]) / h
        A[k, k + 1] = A[k + 1, k] = -arith
        A[k, k] += arith - harm
        A[k + 1, k + 1] += arith - harm
    t_bad = np.linalg.solve(A, P["b"])
    R = np.cumsum(h / kz) - 0.5 * h / kz
    exact = R / np.sum(h / kz)
    assert np.max(np.abs(t_bad - exact)) > 1e-3
    t_ok = np.linalg.solve(P["A"].toarray(), P["b"])
    assert np.max(np.abs(t_ok - exact)) < 1e-12
