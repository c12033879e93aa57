"""Status codes of the C ABI on a GPU (failures made on the host side: bad
arguments and call order; nothing faults the device)."""
import numpy as np
import pytest
import torch

import workloads as W
from helpers import gpu_solver, small_problem
from paper_2410_06850_gb300 import Solver, ThermoError, thermo

pytestmark = pytest.mark.gpu


def test_empty_dirichlet_set_is_rejected():
    grid = (8, 8, 8)
    with pytest.raises(ThermoError) as e:
        Solver(grid, (0.125,) * 3, torch.zeros(9 ** 3, dtype=torch.uint8), torch.ones(512))
    assert e.value.status == thermo.EINVAL


def test_call_order_and_arguments():
    pr = small_problem(8)
    s = Solver(pr["grid"], pr["h"], torch.as_tensor(pr["mask"]), torch.as_tensor(pr["source"]))
    with pytest.raises(ThermoError) as e:
        s.solve()
    assert e.value.status == thermo.ESTATE
    with pytest.raises(ThermoError) as e:
        s.setup_precond()
    assert e.value.status == thermo.ESTATE
    with pytest.raises(ThermoError) as e:
        s.set_density(torch.as_tensor(pr["x"]), 3.0, 0.0, 1.0)
    assert e.value.status == thermo.EINVAL
    s.set_density(torch.as_tensor(pr["x"]), 3.0, 1e-3, 1.0)
    with pytest.raises(ThermoError) as e:
        s.solve()
    assert e.value.status == thermo.ESTATE
    s.setup_precond()
    s.solve()
    s.set_density(torch.as_tensor(pr["x"]), 3.0, 1e-3, 1.0)  # invalidates the preconditioner
    with pytest.raises(ThermoError) as e:
        s.solve()
    assert e.value.status == thermo.ESTATE
    s.close()


def test_max_iter_returns_enotconv_with_last_iterate():
    pr = small_problem(16, kind="chan", kmin=1e-6)
    s = gpu_solver(pr, prec=1, max_iter=3)
    s.setup_precond()
    u, info = s.solve(tol=1e-12, check=False)
    assert info["status"] == thermo.ENOTCONV and info["iters"] == 3
    assert np.isfinite(u.cpu().numpy()).all()
    s.close()


def test_nan_density_reports_breakdown_not_fault():
    pr = small_problem(8)
    pr["x"] = pr["x"].copy()
    pr["x"][5] = np.nan
    s = gpu_solver(pr, prec=0, pc=1, guess=0)
    s.setup_precond()
    u, info = s.solve(tol=1e-8, check=False)
    assert info["status"] in (thermo.EBREAKDOWN, thermo.ENOTCONV)
    s.close()


def test_bad_options_rejected():
    pr = small_problem(16)
    for kw in (dict(block=3), dict(nu_fine=0), dict(nvec=[7, 17])):
        with pytest.raises(ThermoError):
            Solver(pr["grid"], pr["h"], torch.as_tensor(pr["mask"]), torch.as_tensor(pr["source"]), **kw)


def test_stage_wait_time_out_reports_ecuda_and_context_recovers():
    """The bounded waits of the TMA-staged fine kernels (FP32 sweeps, fused
    restriction, float-float and FP64 applies) made to run out on purpose
    through a one-cycle wait limit: every entry point that launched one
    returns ECUDA, the kernels drain their copies and exit, and with the
    default limit restored the same context reproduces its earlier results
    and solves to the oracle's residual."""
    from helpers import oracle_problem
    pr = small_problem(64, kind="chan", seed=3, kmin=1e-6)
    s = gpu_solver(pr, prec=1)
    s.setup_precond()
    n = s.nnode
    rng = np.random.default_rng(11)
    r = torch.as_tensor(rng.standard_normal(n))
    z0 = s.vcycle(r)
    p = torch.as_tensor(rng.standard_normal(n)) * torch.as_tensor(1 - pr["mask"].astype(np.float64))
    q0, d0 = s.apply_dot(p)
    y0 = s.apply(r, thermo.FP64)
    s.set_stage_wait(1)
    for call in (lambda: s.vcycle(r), lambda: s.apply_dot(p), lambda: s.apply(r, thermo.FP64),
                 lambda: s.apply(r, thermo.MIXED), s.setup_precond):
        with pytest.raises(ThermoError) as e:
            call()
        assert e.value.status == thermo.ECUDA, e.value
    s.set_stage_wait(0)
    s.setup_precond()
    assert torch.equal(s.vcycle(r), z0)
    q1, d1 = s.apply_dot(p)
    assert torch.equal(q1, q0) and d1 == d0
    assert torch.equal(s.apply(r, thermo.FP64), y0)
    u, info = s.solve(tol=1e-10)
    assert info["status"] == thermo.OK
    P = oracle_problem(pr)
    res = P["b"] - P["A"] @ u.cpu().numpy()
    assert np.linalg.norm(res) <= 1.5e-10 * np.linalg.norm(P["b"])
    with pytest.raises(ThermoError) as e:
        s.set_stage_wait(-1)
    assert e.value.status == thermo.EINVAL
    s.close()
