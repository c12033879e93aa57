"""Write the FP64 oracle's solution of named workloads at sampled nodes.

    python tests/golden/make_oracle_solutions.py chan128_1e3 chan128_1e6 chan128_1e9

For each workload (``workloads.problem``) this builds the oracle's assembled
Q1 system (Sec. 2.2 Eq. (5)) and its multiscale multigrid hierarchy (Sec. 3,
Eqs. (8)-(9), the default options for N), starts from the interpolated coarse
solution, and runs preconditioned CG (Sec. 4; Algorithm 1 as the
preconditioner):

* to ||b - A u|| <= 1e-13 ||b_F|| for the reference solution u* (or to the
  FP64 floor of the true residual: the solver stops after five residual
  replacements, and the file records the true residual reached);
* to 1e-8 from the same start, for the iteration count the GPU's plain FP64
  form is compared with (same cycle, same stopping rule).

It writes ``tests/golden/oracle_<name>.json``: u* at 4096 nodes drawn by a
seeded partial Fisher-Yates shuffle (stream 41, ``workloads``), the 2-norm,
max-norm and compliance f^T u* of the whole solution, both iteration counts,
the true relative residuals, the wall times and the host.  Only ``oracle/``
and the shared input generator are called: no value here comes from the CUDA
path.  The parity tests and the benchmark read these files.
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import fem, krylov, mmg  # noqa: E402

SAMPLE_SEED = 41
NSAMPLE = 4096


def golden_path(name: str) -> str:
    return os.path.join(HERE, f"oracle_{name}.json")


def solve(name: str) -> dict:
    pr = W.problem(name)
    t0 = time.perf_counter()
    P = fem.build_problem(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], pr["mask"],
                          pr["source"])
    t1 = time.perf_counter()
    H = mmg.MMG(P)
    t2 = time.perf_counter()
    free = ~P["mask"]
    u0 = H.coarse_guess(P["b"])
    u8, i8 = krylov.pcg(P["A"], P["b"], precond=H, u0=u0, tol=1e-8, free=free)
    t3 = time.perf_counter()
    us, ist = krylov.pcg(P["A"], P["b"], precond=H, u0=u0, tol=1e-13, free=free)
    t4 = time.perf_counter()
    n = us.size
    idx = np.sort(W.fisher_yates_sample(SAMPLE_SEED, n, min(NSAMPLE, n)))
    return {
        "name": name, "grid": list(pr["grid"]), "p": pr["p"], "kmin": pr["kmin"], "kmax": pr["kmax"],
        "hierarchy": {"nvec": list(H.opts.nvec), "group": list(H.opts.group), "sizes": H.sizes},
        "solver": "oracle MMG-PCG (standard), coarse initial guess",
        "tol_ref": 1e-13, "iters_ref": ist["iters"], "relres_true_ref": ist["relres_true"],
        "converged_ref": bool(ist["converged"]),
        "tol_count": 1e-8, "iters_1e-8": i8["iters"], "relres_true_1e-8": i8["relres_true"],
        "norm2": float(np.linalg.norm(us)), "norminf": float(np.max(np.abs(us))),
        "compliance": fem.compliance(P["f"], us),
        "err_1e-8_vs_ref": float(np.linalg.norm(u8 - us) / np.linalg.norm(us)),
        "sample_seed": SAMPLE_SEED, "samples": [int(v) for v in idx], "values": [float(v) for v in us[idx]],
        "seconds": {"assemble": t1 - t0, "setup": t2 - t1, "solve_1e-8": t3 - t2, "solve_1e-13": t4 - t3},
        "host": {"machine": platform.machine(), "python": platform.python_version(), "numpy": np.__version__},
    }


def main(names):
    for name in names:
        d = solve(name)
        with open(golden_path(name), "w") as f:
            json.dump(d, f, indent=0)
        import resource
        rss_gb = resource.getrusage(resource.RUSAGE_SELF).ru_maxrss / 2**20
        print(name, d["iters_ref"], d["iters_1e-8"], d["relres_true_ref"], d["seconds"], f"peak RSS {rss_gb:.1f} GB",
              flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
