"""The resolution change of Sec. 3's interpolation technique through the C ABI
(thermo_resample) against the oracle's definition (oracle.topopt.resample,
pinned in tests/test_oracle_resample.py): bit-identical for all three kinds
(both round each product and sum separately in the same order), on ragged
grids, mixed ratios and a grid of many CTAs.  And the physics of the nodal
kind: a 16^3 solution carried to 32^3 is the same function, so the library's
compliance f^T u on the fine grid equals the coarse one, and a fine solve
started from it converges."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import gpu_solver, small_problem
from oracle import fem, topopt
from paper_2410_06850_gb300 import thermo as T

pytestmark = pytest.mark.gpu

CASES = [((3, 2, 4), (6, 4, 8)), ((2, 3, 2), (2, 6, 8)), ((8, 8, 8), (32, 32, 32)), ((64, 48, 32), (128, 96, 64))]


@pytest.mark.parametrize("gc,gf", CASES)
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_resample_bit_identical_to_oracle(gc, gf, kind):
    n = fem.n_nodes(gc) if kind == 2 else gc[0] * gc[1] * gc[2]
    v = W.uniform01(81 + kind, n) - 0.25
    ref = topopt.resample(gc, v, gf, kind)
    out = T.resample(gc, torch.as_tensor(v), gf, kind).cpu().numpy()
    assert out.shape == ref.shape
    assert np.array_equal(out, ref), np.max(np.abs(out - ref))


def test_resample_rejects_bad_arguments():
    v = torch.zeros(64, dtype=torch.float64, device="cuda")
    for gf, kind in [((6, 8, 8), 0), ((8, 8, 8), 3), ((2, 8, 8), 1)]:
        with pytest.raises(T.ThermoError):
            T.resample((4, 4, 4), v, gf, kind)


def test_carried_solution_keeps_compliance_and_warm_starts():
    pc = small_problem(16, kind="smooth", seed=7)
    pf = small_problem(32, kind="smooth", seed=7)
    # the fine design is the coarse one carried piecewise constant: the same conductivity field
    pf["x"] = topopt.resample(pc["grid"], pc["x"], pf["grid"], 0)
    sc = gpu_solver(pc, prec=0)
    sc.setup_precond()
    uc, _ = sc.solve(tol=1e-12)
    uf = T.resample(pc["grid"], uc, pf["grid"], 2)
    sf = gpu_solver(pf, prec=0, guess=1)
    cc, cf = sc.compliance(uc), sf.compliance(uf)
    assert abs(cf - cc) <= 1e-12 * abs(cc), (cf, cc)
    sf.setup_precond()
    u, info = sf.solve(u=uf.clone(), tol=1e-8)
    assert info["rel_res_true"] <= 1e-8, info
    sc.close()
    sf.close()
