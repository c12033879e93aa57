"""Shared test helpers: named small problems for both sides, tolerances."""
import numpy as np

import workloads as W


def small_problem(N, kind="smooth", seed=7, kmin=1e-3, grid=None, h=None, mask="patch"):
    grid = tuple(grid) if grid is not None else (N, N, N)
    M = grid[0] * grid[1] * grid[2]
    if kind == "smooth":
        if grid[0] == grid[1] == grid[2]:
            x = W.smooth_random_density(grid[0], seed)
        else:
            x = 0.05 + 0.95 * W.uniform01(seed, M)
    elif kind == "chan":
        x = W.channel_tree_density(grid[0], seed, 0.2)
    elif kind == "thresh":
        x = W.smoothed_threshold_density(grid[0], seed, 0.3)
    elif kind == "rand":
        x = W.uniform01(seed, M)
    else:
        raise KeyError(kind)
    if isinstance(mask, str):
        m = W.dirichlet_patch_mask(grid) if mask == "patch" else W.full_face_mask(grid, mask)
    else:
        m = mask
    h = tuple(h) if h is not None else tuple(1.0 / g for g in grid)
    return dict(grid=grid, h=h, mask=m, source=W.uniform_source(grid), x=x, p=3.0, kmin=kmin, kmax=1.0)


def oracle_problem(pr):
    from oracle import fem
    return fem.build_problem(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], pr["mask"],
                             pr["source"], pr.get("values"))


def gpu_solver(pr, **opts):
    import torch
    from paper_2410_06850_gb300 import Solver
    s = Solver(pr["grid"], pr["h"], torch.as_tensor(pr["mask"]), torch.as_tensor(pr["source"]),
               dirichlet_value=None if pr.get("values") is None else torch.as_tensor(pr["values"]), **opts)
    s.set_density(torch.as_tensor(pr["x"]), pr["p"], pr["kmin"], pr["kmax"])
    return s


def relerr(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
