"""Hierarchies whose groups are not powers of two.  The paper's sd (coarse
cells per coarse-coarse cell per axis, Sec. 4) takes values such as 6 and 7;
here level 2 groups 3 x 3 x 3 level-1 blocks (27 cells, local problems of
Eq. (9) with 108 unknowns) on a 48^3 grid (12^3 blocks -> 4^3 groups):

* one FP64 cycle equals the oracle's cycle on the library's exported bases to
  1e-11 (the restriction takes its one-thread-per-output path for g^3 = 27);
* FP64 and mixed solves reach the oracle's solution (its own MMG-PCG to 1e-13)
  to 1e-8, the FP64 form within +-2 iterations of the oracle's count."""
import numpy as np
import pytest
import torch

from helpers import gpu_solver, library_bases, oracle_problem, relerr, small_problem
from oracle import krylov, mmg

pytestmark = pytest.mark.gpu

OPTS = dict(levels=2, group=[3], nvec=[4, 17])


def _oracle_opts():
    o = mmg.default_options(48)
    o.nvec = (4, 17)
    o.group = (3,)
    return o


def test_group3_cycle_on_library_bases_matches_oracle():
    pr = small_problem(48, kind="smooth")
    P = oracle_problem(pr)
    s = gpu_solver(pr, prec=0, **OPTS)
    s.setup_precond()
    h = s.hierarchy()
    assert [lv["cells"] for lv in h] == [(12, 12, 12), (4, 4, 4)]
    G = mmg.MMG(P, _oracle_opts(), bases=library_bases(s, pr))
    rng = np.random.default_rng(48)
    for _ in range(2):
        r = rng.standard_normal(P["A"].shape[0])
        r[P["mask"]] = 0.0
        z = s.vcycle(torch.as_tensor(r)).cpu().numpy()
        assert relerr(z, G(r)) < 1e-11, relerr(z, G(r))
    s.close()


@pytest.mark.parametrize("kind,kmin", [("smooth", 1e-3), ("chan", 1e-6)])
def test_group3_solves_match_oracle(kind, kmin):
    pr = small_problem(48, kind=kind, seed=3, kmin=kmin)
    P = oracle_problem(pr)
    H = mmg.MMG(P, _oracle_opts())
    free = ~P["mask"]
    u0 = H.coarse_guess(P["b"])
    _, i8 = krylov.pcg(P["A"], P["b"], precond=H, u0=u0, tol=1e-8, free=free)
    us, _ = krylov.pcg(P["A"], P["b"], precond=H, u0=u0, tol=1e-13, free=free)
    for prec in (0, 1):
        s = gpu_solver(pr, prec=prec, **OPTS)
        s.setup_precond()
        u, info = s.solve(tol=1e-8)
        e = relerr(u.cpu().numpy(), us)
        msg = f"{kind} prec={prec}: iters {info['iters']} (oracle {i8['iters']}), err {e:.2e}"
        assert info["rel_res_true"] <= 1e-8 and e <= 1e-8, msg
        if prec == 0:
            assert abs(info["iters"] - i8["iters"]) <= 2, msg
        s.close()
