"""Benchmark: 256^3 MMG-preconditioned solve to 1e-8 on one GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole path over the synthetic 256^3 workload
(channel-tree density, V = 0.2, contrast 1e6, q = 1, T = 0 on the centred
0.2 x 0.2 patch of z = 0): set_density, setup_precond (local spectral
problems, Galerkin operators, coarsest Cholesky), solve to ||r|| <= 1e-8 ||b||
with the mixed-precision preconditioner (FP32 V-cycle inside FP64 flexible
CG), and the adjoint sensitivity.  `value` is the mean solve time in seconds
(the headline metric); set-up, iterations, the FP64 form and the BF16
smoother variant, per-kernel timings and the roofline of the dominant kernel
are reported beside it.  Inputs are resident in HBM; the working set
(~8 GB per context) is far larger than L2, so no flush is needed.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload family and scales it to the metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "256^3 solve time to 1e-8 (s), iters, DOF/s/apply: mixed vs FP64 on 1 GB300"
WORKLOAD = "chan256_1e6"


FP64_NOMINAL_GFLOPS = 1250.0
# ncu dram__bytes_read.sum + dram__bytes_write.sum per launch of the current kernels at this
# workload (profiles/ summaries); None where no capture of the current kernel exists.
# smooth: the separable three-term sweep, captured on a 192^3 context and scaled by the node count
# (153.45 MB for 7,189,057 nodes); classes made of many kernels (coarse levels) have none
TRAFFIC = {"smooth": 153.45e6 * 16974593 / 7189057, "apply_fp64": None, "coarse_levels": None}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.7), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu=0):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_inputs(name):
    import workloads as W
    return W.problem(name)


def oracle_sample(name):
    """One oracle MMG-PCG solve (FP64, CPU) of a smaller problem of the benchmark's
    family: returns set-up and solve seconds, iterations and node count."""
    import workloads as W
    from oracle import fem, krylov, mmg
    pr = W.problem(name)
    P = fem.build_problem(pr["grid"], pr["h"], pr["x"], pr["p"], pr["kmin"], pr["kmax"], pr["mask"],
                          pr["source"])
    t0 = time.perf_counter()
    H = mmg.MMG(P)
    t1 = time.perf_counter()
    u0 = H.coarse_guess(P["b"])
    _, info = krylov.pcg(P["A"], P["b"], precond=H, u0=u0, tol=1e-8, flexible=True)
    t2 = time.perf_counter()
    n = (pr["grid"][0] + 1) * (pr["grid"][1] + 1) * (pr["grid"][2] + 1)
    return {"setup_s": t1 - t0, "solve_s": t2 - t1, "iters": info["iters"], "nodes": n, "name": name}


def host_info():
    """Host cores and CPU model (the oracle's timings run on these cores)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k = ln.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    import platform
    return {"host_cores": os.cpu_count(), "cpu_model": model or platform.machine()}


def cpu_baseline(iters256, name="chan64"):
    """The oracle as it stands on the host cores.

    * measured: one full oracle run (set-up + MMG-PCG solve to 1e-8) of the
      32^3 configuration (cube32), timed directly;
    * value: a bounded sample of the benchmark's family (channel tree, contrast
      1e6, ``name``) whose solve time is scaled to the 256^3 solve by nodes x
      iterations (seconds per iteration per node x 257^3 x iters256, the FP64
      form's iteration count at 256^3, which the oracle's identical algorithm
      reproduces within two iterations where both run): an extrapolation, said
      so in the line.
    scipy's sparse kernels are single-threaded, so the oracle uses one core."""
    direct = oracle_sample("cube32")
    o = oracle_sample(name)
    n256 = 257 ** 3
    value = o["solve_s"] / max(o["iters"], 1) / o["nodes"] * n256 * iters256
    out = {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
           "sample": (f"oracle MMG-PCG solve of {name} ({o['nodes']} nodes, contrast 1e6): set-up "
                      f"{o['setup_s']:.1f} s (not in value), solve {o['solve_s']:.1f} s, {o['iters']} iterations; "
                      f"extrapolated by nodes x {iters256} iterations to 256^3 (not a 256^3 timing); scipy sparse "
                      f"kernels are single-threaded"),
           "extrapolated": True, "oracle": o,
           "measured": {"workload": "cube32 (32^3, the oracle's full set-up and solve to 1e-8, timed directly)",
                        **direct}}
    out.update(host_info())
    return out


def rank_barrier(dist, cuda=True):
    """Barrier over the replica ranks, then a device synchronisation."""
    if dist is not None:
        dist.barrier()
    if cuda:
        import torch
        torch.cuda.synchronize()


def max_over_ranks(v, dist, device="cuda"):
    """The largest of the ranks' values: the job's time is its slowest replica's."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reference_sample(iters256, name):
    """One reference-arm step: the oracle's set-up and solve of a bounded sample,
    its solve time scaled to 256^3 by nodes x iterations (as cpu_baseline)."""
    o = oracle_sample(name)
    value = o["solve_s"] / max(o["iters"], 1) / o["nodes"] * 257 ** 3 * iters256
    return {"value": value, "sample": (f"oracle MMG-PCG solve of {name} ({o['nodes']} nodes, contrast 1e6): set-up "
                                       f"{o['setup_s']:.1f} s (not in value), solve {o['solve_s']:.1f} s, "
                                       f"{o['iters']} iterations; extrapolated by nodes x {iters256} iterations to "
                                       f"256^3; scipy sparse kernels are single-threaded")}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    K, Wm = args.steps, args.warmup
    vals = []
    last = None
    for i in range(Wm + K):
        cb = reference_sample(args.ref_iters, name="chan48")
        if i >= Wm:
            vals.append(cb["value"])
        last = cb
    v = statistics.mean(vals) if vals else last["value"]
    out = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus, "steps": K, "warmup": Wm,
           "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": "chan256_1e6 (256^3 Q1, channel tree V=0.2, contrast 1e6), sampled at 48^3 "
                                  "and scaled by nodes x iterations", "tol": 1e-8},
           "cpu_baseline": {"value": v, "unit": "s", "kind": "oracle", "cores": 1, "sample": last["sample"],
                            "extrapolated": True, **host_info()},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def loop_hierarchy(grid):
    """Options for a design loop: one set-up per solve, and warm-started solves
    of 15-20 iterations, so the set-up dominates.  Where the default hierarchy
    ends in the exact 8,704-unknown coarsest level (grids above 128 per axis,
    about 1 s of FP64 factorisation per set-up), go one level deeper instead
    (4^3 coarsest cells, 1,088 unknowns, W-cycle): the cheaper set-up."""
    from paper_2410_06850_gb300 import thermo
    o = thermo.default_options(grid)
    L = o.levels
    top = [c // 4 for c in grid]
    for g in list(o.group)[1:L]:
        top = [c // g for c in top]
    if min(top) <= 4 or L >= thermo.MAX_LEVELS:
        return {}
    return dict(levels=L + 1, nvec=list(o.nvec)[:L] + [17], group=list(o.group)[1:L] + [2])


def run_topopt(args, pr, mask_d, q_d):
    """SIMP / optimality-criteria loop on the benchmark geometry: density filter
    radius 1.5 elements, volume fraction 0.3, from uniform x = 0.3; every solve
    starts from the previous solution corrected by the interpolated coarse
    solution (warm coarse guess).  Hierarchy: loop_hierarchy (cheaper set-up)."""
    import torch
    from paper_2410_06850_gb300 import Solver, thermo
    grid = pr["grid"]
    M = grid[0] * grid[1] * grid[2]
    nnode = (grid[0] + 1) * (grid[1] + 1) * (grid[2] + 1)
    p, kmin, kmax, rmin, vf = 3.0, 1e-3, 1.0, 1.5, 0.3
    s = Solver(grid, pr["h"], mask_d, q_d, prec=thermo.MIXED, guess=3, **loop_hierarchy(grid))
    x = torch.full((M,), vf, dtype=torch.float64, device="cuda")
    dv = s.filter(torch.ones(M, dtype=torch.float64, device="cuda"), rmin, transpose=True)
    u = torch.zeros(nnode, dtype=torch.float64, device="cuda")
    hist = []
    torch.cuda.synchronize()
    t_all = time.perf_counter()
    for it in range(args.topopt):
        t0 = time.perf_counter()
        xp = s.filter(x, rmin)
        s.set_density(xp, p, kmin, kmax)
        s.setup_precond()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u, info = s.solve(u=u, tol=args.tol)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        c = s.compliance(u)
        dc = s.filter(s.sensitivity(u), rmin, transpose=True)
        change = s.oc_update(x, dc, dv, vf, 0.2, rmin)
        torch.cuda.synchronize()
        hist.append({"it": it, "compliance": c, "iters": info["iters"], "setup_s": t1 - t0, "solve_s": t2 - t1,
                     "step_s": time.perf_counter() - t0, "change": change, "volume": float(xp.mean())})
    total = time.perf_counter() - t_all
    out = {"mode": "topopt", "workload": args.workload, "design_iterations": args.topopt,
           "total_s": total, "filter_rmin": rmin, "volfrac": vf, "kmin": kmin, "history": hist}
    if args.fd_check:
        # gradient of the compliance with respect to the physical (filtered) density of the final design
        u, _ = s.solve(u=u, tol=1e-12, check=False)
        worst, recs, tfd, nunder = fd_check(s, xp, u, p, kmin, kmax, args.fd_check)
        out["fd_check"] = {"elements": args.fd_check, "seed": 4, "relative_step": 1e-4, "max_rel_err": worst,
                           "target": 1e-6, "checked": args.fd_check - nunder, "sensitivity_underflow": nunder,
                           "seconds": tfd, "records": recs,
                           "what": "adjoint sensitivity vs central differences of c = f^T u formed through the "
                                   "library's operator and solves (no cancellation), final design of the loop"}
    s.close()
    print(json.dumps(out))
    return 0


def run_multires(args):
    """SIMP / OC across resolutions with the interpolation technique of Sec. 3
    (Sec. 4.1: 128^3 -> 256^3 -> 512^3): stage k runs its design iterations on
    an N_k^3 grid; the next stage starts from the design carried by trilinear
    interpolation between cell centres (thermo_resample kind 1) and from the
    solution carried as the same Q1 function (kind 2, warm start).  Same
    harness as --topopt (filter radius 1.5 elements of each grid, V = 0.3,
    q = 1, T = 0 on the centred patch).  For every stage after the first, the
    first solve is also run from the coarse guess alone, so that the carried
    warm start's iteration saving is measured."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import workloads as W
    from paper_2410_06850_gb300 import Solver, thermo

    stages = [tuple(int(v) for v in t.split(":")) for t in args.multires.split(",")]
    p, kmin, kmax, rmin, vf = 3.0, 1e-3, 1.0, 1.5, 0.3
    x = u = None
    prev = None
    out = {"mode": "multires", "stages": [], "filter_rmin": rmin, "volfrac": vf, "kmin": kmin}
    t_all = time.perf_counter()
    for N, iters in stages:
        grid = (N, N, N)
        M = N ** 3
        mask_d = torch.as_tensor(W.dirichlet_patch_mask(grid)).cuda()
        q_d = torch.ones(M, dtype=torch.float64, device="cuda")
        s = Solver(grid, (1.0 / N,) * 3, mask_d, q_d, prec=thermo.MIXED, guess=3, **loop_hierarchy(grid))
        rec = {"N": N, "design_iterations": iters, "history": []}
        if prev is None:
            x = torch.full((M,), vf, dtype=torch.float64, device="cuda")
            u = torch.zeros(s.nnode, dtype=torch.float64, device="cuda")
        else:
            x = thermo.resample(prev, x, grid, 1)
            u = thermo.resample(prev, u, grid, 2)
        dv = s.filter(torch.ones(M, dtype=torch.float64, device="cuda"), rmin, transpose=True)
        t_stage = time.perf_counter()
        for it in range(iters):
            t0 = time.perf_counter()
            xp = s.filter(x, rmin)
            s.set_density(xp, p, kmin, kmax)
            s.setup_precond()
            if it == 0 and prev is not None:
                # the warm coarse guess from u = 0 is the coarse guess alone: the comparison
                _, cold = s.solve(u=torch.zeros_like(u), tol=args.tol)
                rec["first_solve_iters_coarse_guess_only"] = cold["iters"]
            u, info = s.solve(u=u, tol=args.tol)
            c = s.compliance(u)
            dc = s.filter(s.sensitivity(u), rmin, transpose=True)
            change = s.oc_update(x, dc, dv, vf, 0.2, rmin)
            torch.cuda.synchronize()
            if it == 0 and prev is not None:
                rec["first_solve_iters_carried_warm_start"] = info["iters"]
            rec["history"].append({"it": it, "compliance": c, "iters": info["iters"], "change": change,
                                   "step_s": time.perf_counter() - t0})
        rec["stage_s"] = time.perf_counter() - t_stage
        out["stages"].append(rec)
        prev = grid
        s.close()
    out["total_s"] = time.perf_counter() - t_all
    print(json.dumps(out))
    return 0


def fd_check(s, xp, u, p, kmin, kmax, count, seed=4, rel_step=1e-4, tol=1e-10):
    """Central finite differences of the compliance c = f^T u on `count` seeded
    elements (partial Fisher-Yates draw, stream `seed`), against the adjoint
    sensitivity kernel (Sec. 2.3).  For x' = x + d e_e with d = +-rel_step x_e
    (a relative step: the central quotient's truncation error for the SIMP power
    law is then about rel_step^2 / 3 at every x_e) the change of the compliance is
    formed without cancellation:
        c' - c = (u + w)^T r,   r = -(A' - A) u = -dkappa (A_e u),   A' w = r,
    (the same number as c(x') - c(x), which in floating point cancels),
    with A_e u the apply of the library's operator on the single-element
    indicator design (kappa 1 on e, 1e-200 elsewhere) and dkappa the exact
    difference of the SIMP law (expm1 / log1p).  The perturbed designs keep the
    preconditioner of x (thermo_update_density); w is solved to `tol` relative
    to ||r||.  Elements whose sensitivity underflows FP64 (x_e^(p-1) below
    1e-100) are reported apart: both sides are zero there to FP64 range.
    w = dk wh is solved as A' wh = -A_e u, so that the right-hand side keeps the
    scale of A_e u whatever the size of dkappa.
    Returns (largest relative error over the representable elements, records,
    seconds, number of underflowing elements)."""
    import math
    import torch
    import workloads as W
    from paper_2410_06850_gb300 import thermo
    M = xp.numel()
    elems = [int(e) for e in W.fisher_yates_sample(seed, M, count)]
    dc = s.sensitivity(u)
    recs, worst, nunder = [], 0.0, 0
    t0 = time.perf_counter()
    for e in elems:
        xe = float(xp[e])
        g = float(dc[e])
        if xe <= 0.0 or (p - 1.0) * math.log10(xe) < -100.0:
            nunder += 1
            recs.append({"element": e, "x": xe, "adjoint": g, "fd": None, "rel_err": None,
                         "note": "sensitivity below FP64 range"})
            continue
        ind = torch.zeros_like(xp)
        ind[e] = 1.0
        s.update_density(ind, 1.0, 1e-200, 1.0)
        ye = s.apply(u, thermo.FP64)  # A_e u: element e alone, unit conductivity
        d = rel_step * xe
        dcs, its = [], []
        for sg in (1.0, -1.0):
            # kappa(x + sg d) - kappa(x) = (kmax - kmin) x^p ((1 + sg d / x)^p - 1)
            dk = (kmax - kmin) * xe ** p * math.expm1(p * math.log1p(sg * d / xe))
            xq = xp.clone()
            xq[e] += sg * d
            s.update_density(xq, p, kmin, kmax)
            # w = dk wh with A' wh = -A_e u (the right-hand side kept at the scale of A_e u)
            wh, info = s.solve(rhs=-ye, u=torch.zeros_like(u), tol=tol, check=False)
            its.append(info["iters"])
            if info["status"] != thermo.OK:
                its.append(info["status_name"])
            dcs.append(-dk * float(torch.dot(u + dk * wh, ye)))
        fd = (dcs[0] - dcs[1]) / (2.0 * d)
        err = abs(fd - g) / abs(g)
        worst = max(worst, err)
        recs.append({"element": e, "x": xe, "adjoint": g, "fd": fd, "rel_err": err, "iters": its})
    s.update_density(xp, p, kmin, kmax)
    return worst, recs, time.perf_counter() - t0, nunder


def run_compare(args, mask_d, q_d):
    """The 128^3 channel design at contrast 1e6 solved in FP64 to tol by the
    multiscale multigrid PCG, by unpreconditioned CG and by point-Jacobi PCG on
    the same GPU kernels (at most 20,000 iterations; beyond that the solver is
    reported as not converged)."""
    import torch
    from paper_2410_06850_gb300 import Solver, thermo
    if args.compare and args.workload == WORKLOAD:
        args.workload = "chan128"
    pr = make_inputs(args.workload)
    grid = pr["grid"]
    x_d = torch.as_tensor(pr["x"]).cuda()
    res = {}
    for name, pc in (("mmg_pcg", thermo.PC_MMG), ("cg", thermo.PC_NONE), ("jacobi_pcg", thermo.PC_JACOBI)):
        s = Solver(grid, pr["h"], mask_d, q_d, prec=thermo.FP64, pc=pc, max_iter=20000,
                   guess=thermo.GUESS_COARSE if pc == thermo.PC_MMG else thermo.GUESS_ZERO)
        s.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.setup_precond()
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        u, info = s.solve(tol=args.tol, check=False)
        conv = info["status"] == thermo.OK
        res[name] = {"iters": info["iters"], "solve_s": info["t_solve_ms"] / 1e3, "setup_s": ts,
                     "rel_res_true": info["rel_res_true"], "converged": conv,
                     "status": "converged" if conv else "did not converge in 20000 iterations"}
        s.close()
    print(json.dumps({"mode": "compare", "workload": args.workload, "tol": args.tol, "precision": "fp64",
                      "results": res}))
    return 0


def hierarchy_bytes(s, lean):
    """Device bytes of the multilevel hierarchy of a set-up context: Phi, and per
    level the Galerkin tiles, l1 inverses, bases Psi, flags and eigenvalues and
    cycle vectors; the coarsest level's dense operator, inverse and scratch."""
    h = s.hierarchy()
    ts = 4 if lean else 12  # FP32 only, or FP64 + FP32 copies
    nn = (s.grid[0] + 3) * (s.grid[1] + 3) * (((s.grid[0] + 3 + 31) // 32) * 32)
    b = nn * h[0]["nvec"] * ts
    for l, lv in enumerate(h):
        nc = lv["cells"][0] * lv["cells"][1] * lv["cells"][2]
        L = lv["nvec"]
        top = l == len(h) - 1
        b += nc * 27 * L * L * (8 if (top and lean) else (ts if not top else 8))
        b += nc * L * L * ts + nc * L * 9 + nc * L * 4 * (4 if lean else 8)
        if l > 0:
            b += nc * 8 * h[l - 1]["nvec"] * L * ts
    n = h[-1]["ndof"]
    return b + 3 * n * n * 8


def run_large(args):
    """The large configuration: one context at N^3 (default 1024^3) in the lean
    form (FP32 design and hierarchy, FP64 outer vectors), contrast 1e6, channel
    tree at volume fraction 0.1; create, set_density, set-up, one solve to tol
    from the coarse guess, one sensitivity.  Prints one JSON line with the
    times, the iteration count, the true residual, the context's device memory
    (measured and planned) and the hierarchy's share of it."""
    import numpy as np
    import torch
    import __graft_entry__ as ge
    ge.build()
    import workloads as W
    from paper_2410_06850_gb300 import Solver, thermo

    N = args.large
    name = f"chan{N}v10"
    t0 = time.perf_counter()
    pr = W.problem(name)
    grid = pr["grid"]
    t_gen = time.perf_counter() - t0
    opts = dict(lean=1, density_fp32=1)
    plan = thermo.plan_bytes(grid, **opts)
    M = grid[0] * grid[1] * grid[2]
    mask_d = torch.as_tensor(pr["mask"]).cuda()
    q_d = torch.ones(M, dtype=torch.float64, device="cuda")  # q = 1 (uniform source)
    x_d = torch.as_tensor(pr["x"]).cuda()
    del pr["x"], pr["mask"]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with ClockSampler() as clk:
        t0 = time.perf_counter()
        s = Solver(grid, pr["h"], mask_d, q_d, **opts)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        ctx_bytes = free0 - torch.cuda.mem_get_info()[0]
        del mask_d, q_d
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
        s.setup_precond()
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        u = torch.zeros(s.nnode, dtype=torch.float64, device="cuda")
        t0 = time.perf_counter()
        u, info = s.solve(u=u, tol=args.tol)
        torch.cuda.synchronize()
        t_solve = time.perf_counter() - t0
        t0 = time.perf_counter()
        dc = s.sensitivity(u)
        c = s.compliance(u)
        torch.cuda.synchronize()
        t_sens = time.perf_counter() - t0
    peak = torch.cuda.mem_get_info()
    hb = hierarchy_bytes(s, True)
    line = {
        "metric": f"{N}^3 lean-form solve to {args.tol:g} + sensitivity (s)", "value": round(t_solve, 4),
        "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f64 outer / f32 cycle",
        "data": "synthetic", "config": {"workload": name, "grid": list(grid), "contrast": 1e6, "volfrac": 0.1,
                                        "form": "mixed, lean (FP32 hierarchy), FP32 design"},
        "iters": info["iters"], "rel_res_true": info["rel_res_true"], "status": info["status"],
        "seconds": {"generate_inputs_host": round(t_gen, 2), "create": round(t_create, 3),
                    "set_density_setup": round(t_setup, 3), "solve": round(t_solve, 3),
                    "sensitivity_compliance": round(t_sens, 4)},
        "dofs": s.nnode, "compliance": c, "dc_sum": float(dc.sum()),
        "memory_gb": {"context_measured": round(ctx_bytes / 1e9, 2), "context_planned": round(plan / 1e9, 2),
                      "hierarchy": round(hb / 1e9, 2), "hierarchy_budget": 180.0,
                      "device_free_after": round(peak[0] / 1e9, 2), "device_total": round(peak[1] / 1e9, 2)},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def golden(name):
    """The oracle's reference solution of a workload at seeded nodes, if written
    (tests/golden/make_oracle_solutions.py, which calls only the oracle)."""
    p = os.path.join(ROOT, "tests", "golden", f"oracle_{name}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


def err_vs_golden(u, gd):
    """Largest error of u over the golden's sampled nodes, relative to the max-norm
    of the oracle's solution."""
    import torch
    idx = torch.as_tensor(gd["samples"], device=u.device)
    ref = torch.as_tensor(gd["values"], dtype=torch.float64, device=u.device)
    return float(torch.max(torch.abs(u[idx] - ref)) / gd["norminf"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-iters", type=int, default=66,
                    help="iterations of the FP64 solve at 256^3 used to scale the oracle sample (the FP64 form's "
                         "measured count with the default hierarchy)")
    ap.add_argument("--profile-kernel", type=int, default=None,
                    help="only build the workload and launch thermo_bench_kernel(K) three times (for ncu)")
    ap.add_argument("--profile-solve", action="store_true",
                    help="only set up and run one mixed solve inside an NVTX range 'solve' (for ncu)")
    ap.add_argument("--profile-setup", action="store_true",
                    help="only run one warm-up set-up, then one set-up inside an NVTX range 'setup' (for ncu)")
    ap.add_argument("--prec", type=int, default=1, help="precision of the profiling modes")
    ap.add_argument("--no-contrasts", action="store_true", help="skip the contrast 1e3 / 1e9 solves")
    ap.add_argument("--topopt", type=int, default=0,
                    help="run N SIMP/OC design iterations at the workload's size (density filter 1.5, V = 0.3, "
                         "warm-started coarse guesses) and print one JSON line")
    ap.add_argument("--kernels-only", action="store_true", help="only time the kernels and one solve per form")
    ap.add_argument("--fd-check", type=int, default=0,
                    help="with --topopt: central finite differences on N seeded elements of the final design")
    ap.add_argument("--multires", default="",
                    help="SIMP/OC across resolutions, e.g. 128:40,256:20 (N:design iterations per stage)")
    ap.add_argument("--large", type=int, default=0,
                    help="the large configuration at N^3 (1024: the full size) in the lean form; one JSON line")
    ap.add_argument("--compare", action="store_true",
                    help="FP64 MMG-PCG vs CG vs Jacobi-PCG on the workload (default chan128) and print one JSON line")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.large:
        return run_large(args)
    if args.multires:
        return run_multires(args)

    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2410_06850_gb300 import Solver, thermo

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    if args.compare and args.workload == WORKLOAD:
        args.workload = "chan128"
    pr = make_inputs(args.workload)
    grid = pr["grid"]
    nnode = (grid[0] + 1) * (grid[1] + 1) * (grid[2] + 1)
    x_d = torch.as_tensor(pr["x"]).cuda()
    mask_d = torch.as_tensor(pr["mask"]).cuda()
    q_d = torch.as_tensor(pr["source"]).cuda()

    def make(prec):
        s = Solver(grid, pr["h"], mask_d, q_d, prec=prec)
        return s

    def step(s, u):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
        s.setup_precond()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u, info = s.solve(u=u, tol=args.tol)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        dc = s.sensitivity(u)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        return u, dc, info, dict(setup=t1 - t0, solve=t2 - t1, sens=t3 - t2, step=t3 - t0)

    def barrier():
        rank_barrier(dist)

    def maxr(v):
        return max_over_ranks(v, dist)

    if args.kernels_only:
        res = {}
        for prec in (thermo.MIXED, thermo.MIXED_BF16S, thermo.FP64):
            sv = make(prec)
            sv.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
            t0 = time.perf_counter()
            sv.setup_precond()
            torch.cuda.synchronize()
            ts = time.perf_counter() - t0
            u, info = sv.solve(tol=args.tol)
            ks = {}
            for k in range(13):
                try:
                    ms, by = sv.bench_kernel(k, 10)
                    ks[k] = (round(ms, 4), round(by / (ms * 1e-3) / 1e9, 1) if by else None)
                except Exception:
                    pass
            res[prec] = {"setup_s": ts, "iters": info["iters"], "solve_s": info["t_solve_ms"] / 1e3,
                         "rel": info["rel_res_true"], "kernels_ms_GBps": ks}
            sv.close()
        print(json.dumps(res))
        return 0

    if args.topopt:
        return run_topopt(args, pr, mask_d, q_d)
    if args.compare:
        return run_compare(args, mask_d, q_d)

    if args.profile_setup:
        s = make(args.prec)
        s.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
        s.setup_precond()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("setup")
        t0 = time.perf_counter()
        s.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
        s.setup_precond()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print(json.dumps({"setup_s": time.perf_counter() - t0}))
        s.close()
        return 0

    if args.profile_kernel is not None or args.profile_solve:
        s = make(args.prec)
        s.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
        if args.profile_kernel is None or args.profile_kernel in (4, 5, 6, 8, 9):
            s.setup_precond()
        if args.profile_kernel is not None:
            ms, by = s.bench_kernel(args.profile_kernel, 3)
            print(json.dumps({"kernel": args.profile_kernel, "ms": ms, "bytes": by}))
        else:
            s.solve(tol=args.tol)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("solve")
            u, info = s.solve(tol=args.tol)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
            print(json.dumps({"iters": info["iters"], "solve_ms": info["t_solve_ms"]}))
        s.close()
        return 0

    # ---- mixed form (headline)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    s = make(thermo.MIXED)
    s.set_density(x_d, pr["p"], pr["kmin"], pr["kmax"])
    s.setup_precond()
    torch.cuda.synchronize()
    footprint_gb = (free0 - torch.cuda.mem_get_info()[0]) / 1e9
    u = torch.zeros(nnode, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        u, dc, info, tm = step(s, u)
    barrier()
    # per-kernel-class CUDA-event timers on the context stream, live over the timed steps
    s.kernel_timers(True)
    l0 = thermo.launch_count()
    times, infos = [], []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            u, dc, info, tm = step(s, u)
            times.append(tm)
            infos.append(info)
        barrier()
    launches = thermo.launch_count() - l0
    klass = {}
    for kc, kn in thermo.KT_NAMES.items():
        ms, nl, by, fl = s.kernel_time(kc)
        klass[kn] = {"ms_total": ms, "launches": nl, "ms_per_launch": ms / nl if nl else None,
                     "bytes_per_launch": by / nl if nl else None, "flops_per_launch": fl / nl if nl else None}
    s.kernel_timers(False)
    solve_s = maxr(statistics.mean(t["solve"] for t in times))
    step_s = maxr(statistics.mean(t["step"] for t in times))
    setup_s = statistics.mean(t["setup"] for t in times)
    sens_s = statistics.mean(t["sens"] for t in times)
    iters = infos[-1]["iters"]

    # ---- per-kernel timings (same context, CUDA events on its stream)
    s.bench_kernel(7, 1)
    kern = {}
    names = {0: "apply_fp64", 1: "apply_fp32", 3: "smooth_fp32", 4: "restrict_fp32", 5: "prolong_smooth_fp32",
             6: "level1_apply_fp32", 7: "cg_update_fp64", 8: "vcycle_mixed"}
    for k, nm in names.items():
        ms, by = s.bench_kernel(k, 20)
        kern[nm] = {"ms": ms, "bytes": by, "GBps": (by / (ms * 1e-3) / 1e9) if by else None}
    hbm, peak_kind = _peaks()
    dof_apply = {"fp64": nnode / (kern["apply_fp64"]["ms"] * 1e-3),
                 "fp32": nnode / (kern["apply_fp32"]["ms"] * 1e-3)}

    # ---- e2e: the same solve through the public API from HOST buffers (pinned):
    # H2D of the right-hand side, thermo_solve, D2H of the solution, all timed
    b_h = s.load_vector().cpu().pin_memory()
    u_h = torch.empty(nnode, dtype=torch.float64).pin_memory()
    e2e = []
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bd = b_h.cuda(non_blocking=True)
        uu, inf2 = s.solve(rhs=bd, tol=args.tol)
        u_h.copy_(uu, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    e2e_s = maxr(statistics.median(e2e))
    e2e_iters = inf2["iters"]

    # ---- BF16-smoother variant and the plain FP64 form
    variants = {}
    for nm, prec in (("mixed_bf16s", thermo.MIXED_BF16S), ("fp64_form", thermo.FP64)):
        sv = make(prec)
        uv = torch.zeros(nnode, dtype=torch.float64, device="cuda")
        uv, _, iv, tv = step(sv, uv)  # warm-up
        ts = []
        for _ in range(max(1, min(args.steps, 2))):
            uv, _, iv, tv = step(sv, uv)
            ts.append(tv)
        variants[nm] = {"solve_s": statistics.mean(t["solve"] for t in ts),
                        "setup_s": statistics.mean(t["setup"] for t in ts), "iters": iv["iters"],
                        "rel_res_true": iv["rel_res_true"],
                        "rel_diff_vs_mixed": float(torch.linalg.norm(uv - u) / torch.linalg.norm(u))}
        if prec == thermo.MIXED_BF16S:
            ms, by = sv.bench_kernel(2, 20)
            kern["apply_bf16"] = {"ms": ms, "bytes": by, "GBps": by / (ms * 1e-3) / 1e9}
            dof_apply["bf16"] = nnode / (ms * 1e-3)
        if prec == thermo.FP64:
            for k, kn in ((9, "vcycle_fp64"), (10, "smooth_fp64")):
                ms, by = sv.bench_kernel(k, 10)
                kern[kn] = {"ms": ms, "bytes": by, "GBps": (by / (ms * 1e-3) / 1e9) if by else None}
        sv.close()

    # ---- contrast sweep: the same geometry at kmin = 1e-3 and 1e-9 (mixed form and the FP64 form), each
    # solution's error against the oracle's reference solution where it has been written (tests/golden)
    contrasts = {}
    if not args.no_contrasts and args.workload == WORKLOAD:
        def solve_pair(pc_, tag_golden):
            xc = torch.as_tensor(pc_["x"]).cuda()
            gd = golden(tag_golden)
            res = {}
            for tag, prec in (("mixed", thermo.MIXED), ("fp64_form", thermo.FP64)):
                sv = Solver(pc_["grid"], pc_["h"], torch.as_tensor(pc_["mask"]).cuda(),
                            torch.as_tensor(pc_["source"]).cuda(), prec=prec)
                sv.set_density(xc, pc_["p"], pc_["kmin"], pc_["kmax"])
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sv.setup_precond()
                torch.cuda.synchronize()
                ts = time.perf_counter() - t0
                uc, ic = sv.solve(tol=args.tol)
                uc, ic = sv.solve(tol=args.tol)
                res[tag] = {"solve_s": ic["t_solve_ms"] / 1e3, "iters": ic["iters"], "rel_res_true": ic["rel_res_true"],
                            "setup_s": ts}
                if gd is not None:
                    res[tag]["err_vs_oracle"] = err_vs_golden(uc, gd)
                sv.close()
            d = {"kmin": pc_["kmin"], "mixed": res["mixed"], "fp64_form": res["fp64_form"]}
            if gd is not None:
                d["oracle"] = {"iters_1e-8": gd["iters_1e-8"], "reference_tol": gd["tol_ref"],
                               "reference_rel_res_true": gd["relres_true_ref"], "samples": len(gd["samples"]),
                               "err": "max over the sampled nodes of |u - u*| / max|u*|"}
            else:
                d["oracle"] = "no reference solution written for this workload"
            return d
        for nm in ("chan256_1e3", "chan256_1e9"):
            contrasts[nm] = solve_pair(make_inputs(nm), nm)
        gd = golden(WORKLOAD)
        if gd is not None:
            contrasts[WORKLOAD] = {"kmin": pr["kmin"], "mixed": {"iters": iters, "err_vs_oracle": err_vs_golden(u, gd)},
                                   "oracle": {"iters_1e-8": gd["iters_1e-8"], "reference_tol": gd["tol_ref"],
                                              "reference_rel_res_true": gd["relres_true_ref"]}}
        for nm in ("chan128_1e3", "chan128_1e6", "chan128_1e9"):
            contrasts[nm] = solve_pair(make_inputs(nm), nm)

    # roofline of the dominant kernel class of the timed solves (largest summed event time)
    dom = max(klass, key=lambda k: klass[k]["ms_total"])
    dk = klass[dom]
    if dom == "apply_fp64":
        # FP64 ALU bound: algorithmic flops (2 per stored-matrix nonzero of the row) against the
        # nominal FP64 rate (no measured FP64 peak is available)
        ach = dk["flops_per_launch"] / (dk["ms_per_launch"] * 1e-3) / 1e9
        roof = {"kernel": "fine FP64 Q1 apply + fused p.Ap (CG loop)", "bound": "alu", "achieved": ach,
                "peak": FP64_NOMINAL_GFLOPS, "unit": "GFLOP/s", "frac": ach / FP64_NOMINAL_GFLOPS,
                "peak_kind": "nominal FP64 (recipe table), no measured FP64 peak",
                "hbm_frac": dk["bytes_per_launch"] / (dk["ms_per_launch"] * 1e-3) / 1e9 / hbm}
    else:
        ach = dk["bytes_per_launch"] / (dk["ms_per_launch"] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                "peak_kind": peak_kind}
    roof.update({"traffic": TRAFFIC.get(dom), "class": dom,
                 "ms_per_launch": dk["ms_per_launch"], "launches_timed": dk["launches"],
                 "share_of_solve": dk["ms_total"] / (solve_s * 1e3 * args.steps)})

    out = {"metric": METRIC, "value": solve_s, "unit": "s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
           "config": {"workload": f"{args.workload}: 256^3 Q1 elements (16,974,593 nodes), channel-tree density "
                                  "V=0.2, p=3, kmin=1e-6, kmax=1, q=1, T=0 on 0.2x0.2 patch of z=0",
                      "tol": args.tol, "hierarchy": s.hierarchy(), "l2": "inputs larger than L2 (no flush)",
                      "hbm_footprint_gb": footprint_gb,
                      "parallelism": f"replicas x{world}"},
           "iters": iters, "rel_res_true": infos[-1]["rel_res_true"], "setup_s": setup_s,
           "sensitivity_s": sens_s, "dof_per_s_apply": dof_apply, "variants": variants, "kernels": kern,
           "roofline": roof, "gpu_launches": launches, "kernel_classes": klass, "contrasts": contrasts,
           "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(b_h.numel() * 8),
                   "d2h_bytes_per_step": int(u_h.numel() * 8), "iters": e2e_iters,
                   "what": "H2D right-hand side (pinned) + thermo_solve + D2H solution"},
           "clocks": clk.summary()}
    s.close()
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(variants["fp64_form"]["iters"])
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
