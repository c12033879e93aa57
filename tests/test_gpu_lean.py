"""The lean form (opt.lean: the hierarchy stored once, in FP32) through the
C ABI.

* Device memory: a context takes what thermo_plan_bytes says (within the CUDA
  allocator's rounding) for the default, lean and FP64 forms.
* Level 1 is built by the same FP64 kernels in both forms and rounded once in
  the lean one: its exported Phi and tiles are exactly the FP32 roundings of
  the default form's.
* Solutions: lean and default mixed solves agree (both within 1e-8 of the
  same system's solution), with and without Dirichlet values, and with the
  design given in FP32; the sensitivities of Sec. 2.3 agree.
Solution parity against the oracle at three contrasts is in
tests/test_gpu_parity_scale.py (form mixed_lean)."""
import numpy as np
import pytest
import torch

from helpers import gpu_solver, small_problem
from paper_2410_06850_gb300 import Solver, thermo as T

pytestmark = pytest.mark.gpu


def _context_bytes(pr, **opts):
    dev = torch.device("cuda")
    mask = torch.as_tensor(pr["mask"]).to(dev)
    src = torch.as_tensor(pr["source"]).to(dev)
    dval = None if pr.get("values") is None else torch.as_tensor(pr["values"]).to(dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = Solver(pr["grid"], pr["h"], mask, src, dirichlet_value=dval, **opts)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    s.close()
    return used


@pytest.mark.parametrize("form", [dict(), dict(lean=1, density_fp32=1), dict(prec=0)],
                         ids=["mixed", "lean", "fp64"])
def test_footprint_matches_plan(form):
    pr = small_problem(128, kind="chan", seed=3, kmin=1e-6)
    _context_bytes(small_problem(32), **form)  # loads the kernels' modules first
    used = _context_bytes(pr, **form)
    plan = T.plan_bytes(pr["grid"], **form)
    # cudaMalloc rounds each buffer up to its page size (2 MiB for the large ones)
    assert 0.97 * plan - 64e6 <= used <= 1.03 * plan + 256e6, (used / 1e9, plan / 1e9)


def test_level1_is_the_rounded_default():
    pr = small_problem(32, kind="smooth", seed=7)
    a = gpu_solver(pr)
    b = gpu_solver(pr, lean=1)
    a.setup_precond()
    b.setup_precond()
    h = a.hierarchy()[0]
    ncell = h["cells"][0] * h["cells"][1] * h["cells"][2]
    counts = {0: a.nnode * h["nvec"], 1: ncell * 27 * h["nvec"] ** 2}
    for what in (0, 1):  # Phi, tiles
        xa = a.export_level(1, what, counts[what]).cpu()
        xb = b.export_level(1, what, counts[what]).cpu()
        assert torch.equal(xa.float().double(), xb), what
    a.close()
    b.close()


@pytest.mark.parametrize("case", ["patch", "values", "fp32_design"])
def test_lean_solution_and_sensitivity_match_default(case):
    pr = small_problem(64, kind="chan", seed=3, kmin=1e-6)
    lean_opts = dict(lean=1)
    if case == "values":
        # T_D = 0.3 + 0.1 sin(x) on the patch
        N = pr["grid"][0]
        xs = np.arange(N + 1) / N
        v = np.zeros((N + 1,) * 3)
        v[:, :, :] = 0.3 + 0.1 * np.sin(xs)[None, None, :]
        pr = dict(pr, values=(v.reshape(-1) * pr["mask"]).astype(np.float64))
    a = gpu_solver(pr)
    if case == "fp32_design":
        lean_opts["density_fp32"] = 1
        from paper_2410_06850_gb300 import Solver as S
        b = S(pr["grid"], pr["h"], torch.as_tensor(pr["mask"]), torch.as_tensor(pr["source"]), **lean_opts)
        b.set_density(torch.as_tensor(pr["x"]).float(), pr["p"], pr["kmin"], pr["kmax"])
    else:
        b = gpu_solver(pr, **lean_opts)
    a.setup_precond()
    b.setup_precond()
    ua, ia = a.solve(tol=1e-10)
    ub, ib = b.solve(tol=1e-10)
    e = float(torch.linalg.norm(ua - ub) / torch.linalg.norm(ua))
    msg = f"{case}: iters default {ia['iters']} lean {ib['iters']}, rel diff {e:.2e}"
    assert ib["rel_res_true"] <= 1e-10, msg
    assert e <= 1e-9, msg
    assert ib["iters"] <= ia["iters"] + 3, msg
    da = a.sensitivity(ua)
    db = b.sensitivity(ub)
    ed = float(torch.linalg.norm(da - db) / torch.linalg.norm(da))
    assert ed <= 1e-8, (msg, ed)
    a.close()
    b.close()
