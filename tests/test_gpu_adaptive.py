"""Adaptive local bases (opt.eig_threshold = tau: a cell keeps its local
eigenpairs with lambda H^2 <= tau, at most nvec, at least one) through the C
ABI against the oracle (mmg.kept_count, pinned in tests/test_oracle_mmg.py by
the component count of a high-contrast block):

* the number of active vectors of every cell on every level equals the
  oracle's (read from the exported bases: an inactive slot is a zero column);
  tau = 1 sits in the spectral gap of the binary high-contrast designs (near-
  zero eigenvalues per conductive component, the rest above about 5 / H^2),
  so the integer decisions are not close calls;
* the three-inclusion block keeps three vectors, void blocks one;
* FP64-form solves with the adaptive hierarchy reach the reference solution
  (a direct solve at 32^3, the oracle's MMG-PCG to 1e-13 at 64^3) to 1e-8, with
  the oracle's adaptive MMG-PCG iteration count within +-2.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

import workloads as W
from helpers import gpu_solver
from oracle import fem, krylov, mmg

pytestmark = pytest.mark.gpu


def _lib_counts(s):
    """Active slots per cell of every level, from the exported bases."""
    h = s.hierarchy()
    out = []
    b = 4
    N = s.grid
    for l, lv in enumerate(h, start=1):
        L = lv["nvec"]
        nc = lv["cells"][0] * lv["cells"][1] * lv["cells"][2]
        if l == 1:
            phi = s.export_level(1, 0, s.nnode * L).cpu().numpy().reshape(N[2] + 1, N[1] + 1, N[0] + 1, L)
            nb = [n // b for n in N]
            bi = [np.minimum(np.arange(n + 1) // b, m - 1) for n, m in zip(N, nb)]
            cell = (bi[0][None, None, :] + nb[0] * (bi[1][None, :, None] + nb[1] * bi[2][:, None, None])).ravel()
            nz = (phi.reshape(-1, L) != 0.0)
            act = np.zeros((nc, L), dtype=bool)
            np.logical_or.at(act, cell, nz)
        else:
            Lp = h[l - 2]["nvec"]
            g = round((h[l - 2]["cells"][0] // lv["cells"][0]))
            psi = s.export_level(l, 0, nc * g ** 3 * Lp * L).cpu().numpy().reshape(nc, g ** 3 * Lp, L)
            act = (psi != 0.0).any(axis=1)
        out.append(act.sum(axis=1))
    return out


def _oracle(pr, tau, prec_opts=None):
    P = fem.build_problem(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], pr["mask"], pr["source"])
    o = mmg.default_options(pr["grid"][0])
    o.eig_threshold = tau
    return P, mmg.MMG(P, o)


@pytest.mark.parametrize("name", ["chan32", "chan64"])
def test_adaptive_counts_match_oracle(name):
    pr = W.problem(name)
    P, H = _oracle(pr, 1.0)
    s = gpu_solver(pr, prec=0, eig_threshold=1.0)
    s.setup_precond()
    lib = _lib_counts(s)
    ref = [lev.active.reshape(-1, lev.L).sum(axis=1) for lev in H.levels]
    assert len(lib) == len(ref)
    for l, (a, b) in enumerate(zip(lib, ref), start=1):
        assert np.array_equal(a, b), (l, np.flatnonzero(a != b)[:10], a[a != b][:10], b[a != b][:10])
    # the adaptive hierarchy is smaller than the fixed one on the binary design
    assert lib[0].sum() < lib[0].size * s.hierarchy()[0]["nvec"]
    s.close()


def test_inclusions_block_keeps_one_vector_per_component():
    N = 8
    x = np.zeros((N, N, N))
    for (ex, ey, ez) in [(0, 0, 0), (2, 0, 0), (0, 2, 2)]:
        x[ez, ey, ex] = 1.0
    grid = (N, N, N)
    pr = dict(grid=grid, h=(1.0 / N,) * 3, mask=W.dirichlet_patch_mask(grid), source=W.uniform_source(grid),
              x=x.ravel(), p=3.0, kmin=1e-6, kmax=1.0)
    s = gpu_solver(pr, prec=0, levels=1, nvec=[6], eig_threshold=1.0)
    s.setup_precond()
    c = _lib_counts(s)[0]
    assert c[0] == 3 and np.all(c[1:] == 1), c
    s.close()


@pytest.mark.parametrize("name", ["chan32", "chan64"])
def test_adaptive_solve_matches_direct_and_oracle_iterations(name):
    pr = W.problem(name)
    P, H = _oracle(pr, 1.0)
    free = ~P["mask"]
    u0 = H.coarse_guess(P["b"])
    _, info_or = krylov.pcg(P["A"], P["b"], precond=H, u0=u0, tol=1e-8, free=free)
    if name == "chan32":
        ud = spla.spsolve(P["A"].tocsc(), P["b"])
    else:  # the oracle's own MMG-PCG to its FP64 floor (a sparse direct solve takes minutes here)
        ud, _ = krylov.pcg(P["A"], P["b"], precond=H, u0=u0, tol=1e-13, free=free)
    s = gpu_solver(pr, prec=0, eig_threshold=1.0)
    s.setup_precond()
    u, info = s.solve(tol=1e-10)
    e = np.linalg.norm(u.cpu().numpy() - ud) / np.linalg.norm(ud)
    assert e <= 1e-8, e
    _, i8 = s.solve(tol=1e-8)
    assert abs(i8["iters"] - info_or["iters"]) <= 2, (i8["iters"], info_or["iters"])
    s.close()
