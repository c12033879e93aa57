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


def library_bases(s, pr):
    """The library's coarse spaces as sparse prolongations in the oracle's
    numbering (for oracle.mmg.MMG(..., bases=...)): level 1 Phi (n0 x n1,
    column block * L_1 + j, natural node rows, Dirichlet rows empty) and, per
    level l >= 2, Psi (n_{l-1} x n_l, rows previous-level cell * L_{l-1} + j,
    columns group * L_l + k), rebuilt from thermo_export_level's layouts."""
    import scipy.sparse as sp
    from oracle import mmg
    h = s.hierarchy()
    n0 = s.nnode
    L1 = h[0]["nvec"]
    phi = s.export_level(1, 0, n0 * L1).cpu().numpy().reshape(n0, L1)
    blk, _ = mmg.node_blocks(pr["grid"], 4, pr["mask"])
    rows = np.repeat(np.flatnonzero(blk >= 0), L1)
    free = blk >= 0
    cols = (blk[free][:, None] * L1 + np.arange(L1)[None, :]).reshape(-1)
    vals = phi[free].reshape(-1)
    out = [sp.csr_matrix((vals, (rows, cols)), shape=(n0, h[0]["ndof"]))]
    for l in range(1, len(h)):
        mx, my, mz = h[l - 1]["cells"]
        sx, sy, sz = h[l]["cells"]
        g = mx // sx
        Lp, L = h[l - 1]["nvec"], h[l]["nvec"]
        ncell = sx * sy * sz
        psi = s.export_level(l + 1, 0, ncell * g ** 3 * Lp * L).cpu().numpy().reshape(ncell, g ** 3 * Lp, L)
        G = np.arange(ncell)
        Gx, Gy, Gz = G % sx, (G // sx) % sy, G // (sx * sy)
        loc = np.arange(g ** 3)
        lx, ly, lz = loc % g, (loc // g) % g, loc // (g * g)
        cell = (Gx[:, None] * g + lx[None, :]) + mx * ((Gy[:, None] * g + ly[None, :]) + my * (Gz[:, None] * g + lz[None, :]))
        prow = (cell[:, :, None] * Lp + np.arange(Lp)[None, None, :]).reshape(ncell, g ** 3 * Lp)
        r = np.repeat(prow[:, :, None], L, axis=2).reshape(-1)
        c = np.broadcast_to((G[:, None] * L + np.arange(L)[None, :])[:, None, :], psi.shape).reshape(-1)
        out.append(sp.csr_matrix((psi.reshape(-1), (r, c)), shape=(mx * my * mz * Lp, ncell * L)))
    return out
