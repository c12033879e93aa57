"""The large configuration at full size: 1024^3 elements (1,076,890,625
nodes), channel-tree design at volume fraction 0.1 given in FP32, contrast
1e6, q = 1, T = 0 on the centred patch, in the lean context form (FP32
hierarchy, FP64 outer CG), as `bench.py --large 1024` runs it.  One solve to
1e-8 from the coarse guess and one sensitivity, checked against the oracle
where it can evaluate outputs one by one (Sec. 2.2 Eq. (5) row by row from the
element matrices; Sec. 2.3 element by element):

* the solver's own FP64 true residual <= 1e-8, T = 0 on Gamma_D;
* residual rows b_i - (A u)_i evaluated by the oracle on 30,000 sampled nodes
  (every node of a few tile-edge lines and seeded random nodes): each row is
  within the 2-norm bound ||r|| <= 1e-8 ||b|| (||b|| estimated from the
  sample), and the sampled estimate of ||r|| / ||b|| is <= 2e-8;
* the sensitivity on 4,096 seeded elements (half solid, half void) within
  1e-12 of the oracle's formula applied to the same u, relative to the scale
  p x^(p-1) (kmax - kmin) sum_ab |K0_ab| |u_a| |u_b| of its rounding;
* the context's device memory within 1% of thermo_plan_bytes.
About two minutes on one GB300 and 40 GB of host memory."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import fem
from paper_2410_06850_gb300 import Solver, thermo as T

pytestmark = pytest.mark.gpu

N = 1024


@pytest.fixture(scope="module")
def large():
    torch.cuda.empty_cache()
    pr = W.problem(f"chan{N}v10")
    grid = pr["grid"]
    M = grid[0] * grid[1] * grid[2]
    opts = dict(lean=1, density_fp32=1)
    need = T.plan_bytes(grid, **opts)
    free = torch.cuda.mem_get_info()[0]
    if free < need + 16e9:
        pytest.skip(f"needs {need / 1e9:.0f} GB + inputs on the device, {free / 1e9:.0f} GB free")
    mask_d = torch.as_tensor(pr["mask"]).cuda()
    q_d = torch.ones(M, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = Solver(grid, pr["h"], mask_d, q_d, **opts)
    torch.cuda.synchronize()
    used = free0 - torch.cuda.mem_get_info()[0]
    del mask_d, q_d
    s.set_density(torch.as_tensor(pr["x"]).cuda(), pr["p"], pr["kmin"], pr["kmax"])
    s.setup_precond()
    u, info = s.solve(tol=1e-8)
    dc = s.sensitivity(u)
    res = dict(pr=pr, info=info, used=used, plan=need, u=u.cpu().numpy())
    e_solid = np.flatnonzero(pr["x"] > 0.5)
    e_void = np.flatnonzero(pr["x"] <= 0.5)
    pick = lambda a, seed: a[W.fisher_yates_sample(seed, a.size, 2048)]
    elems = np.concatenate([pick(e_solid, 61), pick(e_void, 62)])
    res["elems"] = elems
    res["dc"] = dc[torch.as_tensor(elems, device=dc.device)].cpu().numpy()
    s.close()
    del u, dc
    torch.cuda.empty_cache()
    return res


def test_memory_matches_plan(large):
    assert abs(large["used"] - large["plan"]) <= 0.01 * large["plan"], (large["used"] / 1e9, large["plan"] / 1e9)


def test_solver_true_residual(large):
    info, pr, u = large["info"], large["pr"], large["u"]
    assert info["status"] == 0 and info["rel_res_true"] <= 1e-8, info
    assert np.all(u[pr["mask"].astype(bool)] == 0.0)


def test_residual_rows_evaluated_by_the_oracle(large):
    pr, u = large["pr"], large["u"]
    g, h = pr["grid"], pr["h"]
    Nx, Ny, Nz = g
    nx, ny, nz = Nx + 1, Ny + 1, Nz + 1
    n = nx * ny * nz
    xs = np.array([0, 1, 31, 32, 511, 512, Nx - 1, Nx])
    ys = np.array([0, 7, 8, 512, Ny])
    zs = np.arange(0, nz, 7)
    zz, yy, xx = np.meshgrid(zs, ys, xs, indexing="ij")
    rnd = np.minimum((W.uniform01(63, 20000) * n).astype(np.int64), n - 1)
    rows = np.unique(np.concatenate([(xx + nx * (yy + ny * zz)).ravel(), rnd]))
    kap = fem.simp_kappa(pr["x"], pr["p"], pr["kmin"], pr["kmax"])
    mask = pr["mask"]
    Au = fem.operator_rows(g, h, kap, mask, u, rows)
    b = np.where(mask[rows].astype(bool), 0.0, fem.load_rows(g, h, 1.0, rows))
    r = b - Au
    # ||b|| and ||r|| estimated from the uniform random part of the sample
    rr = np.isin(rows, rnd)
    bnorm = np.sqrt(n / rr.sum() * np.sum(b[rr] ** 2))
    est = np.sqrt(np.sum(r[rr] ** 2) / np.sum(b[rr] ** 2))
    msg = f"iters {large['info']['iters']}, max |r_i| / ||b|| {np.max(np.abs(r)) / bnorm:.2e}, estimate {est:.2e}"
    assert np.max(np.abs(r)) <= 1.1e-8 * bnorm, msg
    assert est <= 2e-8, msg


def test_sensitivity_elements_evaluated_by_the_oracle(large):
    pr, u, e = large["pr"], large["u"], large["elems"]
    g, h = pr["grid"], pr["h"]
    xe = pr["x"][e].astype(np.float64)
    ref = fem.sensitivity_at(g, h, xe, pr["p"], pr["kmin"], pr["kmax"], u, e)
    absu = np.abs(u)
    K0 = fem.element_matrix(h)
    # rounding scale: the element energy with |K0| and |u|
    Nx, Ny, _ = g
    nx, ny = Nx + 1, Ny + 1
    ex, ey, ez = e % Nx, (e // Nx) % Ny, e // (Nx * Ny)
    base = ex + nx * (ey + ny * ez)
    ue = np.stack([absu[base + (a & 1) + nx * (((a >> 1) & 1) + ny * (a >> 2))] for a in range(8)], axis=1)
    scale = pr["p"] * xe ** (pr["p"] - 1.0) * (pr["kmax"] - pr["kmin"]) * np.einsum("ea,ab,eb->e", ue, np.abs(K0), ue)
    err = np.abs(large["dc"] - ref) / np.maximum(scale, 1e-300)
    assert np.all(large["dc"][pr["x"][e] <= 0.5] == 0.0)  # x = 0: zero sensitivity (p > 1)
    assert err.max() <= 1e-12, err.max()
