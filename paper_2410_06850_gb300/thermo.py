"""ctypes binding of libthermo (argument marshalling only).

Every numerical step runs in libthermo's CUDA kernels; this module passes
device pointers of torch tensors and the current CUDA stream through the C
ABI declared in include/thermo.h.  Importing works without a GPU; any call
that needs the library raises if libthermo.so is missing (no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libthermo.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, EBREAKDOWN, ESINGULAR, ESTATE = 0, -1, -2, -3, -4, -5, -6, -7
FP64, MIXED, MIXED_BF16S = 0, 1, 2
PC_MMG, PC_NONE, PC_JACOBI = 0, 1, 2
GUESS_ZERO, GUESS_GIVEN, GUESS_COARSE, GUESS_WARM_COARSE = 0, 1, 2, 3
MAX_LEVELS = 8
KT_APPLY64, KT_SMOOTH, KT_RESTRICT, KT_PROLONG, KT_COARSE, KT_CGVEC = range(6)
KT_NAMES = {KT_APPLY64: "apply_fp64", KT_SMOOTH: "smooth", KT_RESTRICT: "restrict", KT_PROLONG: "prolong",
            KT_COARSE: "coarse_levels", KT_CGVEC: "cg_vector"}
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENOTCONV",
                -5: "EBREAKDOWN", -6: "ESINGULAR", -7: "ESTATE"}

EXPORTED = ["thermo_default_options", "thermo_create", "thermo_set_density", "thermo_setup_precond",
            "thermo_solve", "thermo_sensitivity", "thermo_compliance", "thermo_last_error",
            "thermo_destroy", "thermo_apply", "thermo_vcycle", "thermo_load_vector",
            "thermo_hierarchy", "thermo_export_level", "thermo_filter", "thermo_oc_update",
            "thermo_launch_count", "thermo_bench_kernel", "thermo_apply_dot",
            "thermo_kernel_timers", "thermo_kernel_time", "thermo_dot_noalloc", "thermo_residual_history",
            "thermo_set_stage_wait", "thermo_dense_spd_inverse", "thermo_update_density",
            "thermo_plan_bytes", "thermo_resample", "thermo_tpfa_conductivity", "thermo_tpfa_apply",
            "thermo_tpfa_rhs", "thermo_tpfa_sensitivity"]


class thermo_options(C.Structure):
    _fields_ = [("levels", C.c_int), ("block", C.c_int), ("group", C.c_int * MAX_LEVELS),
                ("nvec", C.c_int * MAX_LEVELS), ("nu_fine", C.c_int), ("nu_coarse", C.c_int),
                ("omega", C.c_double), ("prec", C.c_int), ("pc", C.c_int), ("guess", C.c_int),
                ("max_iter", C.c_int), ("flexible", C.c_int), ("check_every", C.c_int),
                ("smoother", C.c_int), ("cheb_degree", C.c_int), ("cheb_ratio", C.c_double),
                ("power_iters", C.c_int), ("outer_apply", C.c_int),
                ("nu_growth", C.c_int), ("w_from", C.c_int), ("restart_decades", C.c_double),
                ("density_fp32", C.c_int), ("fine_engine", C.c_int), ("lean", C.c_int),
                ("eig_threshold", C.c_double)]


class thermo_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("rel_res_recursive", C.c_double),
                ("rel_res_true", C.c_double), ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("status", C.c_int)]

    def asdict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ThermoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib_handle = None


def lib():
    """Load libthermo.so (raises if it has not been built)."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2410_06850_gb300.build`")
        L = C.CDLL(LIB_PATH)
        vp, ip, dp, i = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int
        L.thermo_default_options.argtypes = [ip, C.POINTER(thermo_options)]
        L.thermo_create.argtypes = [ip, dp, vp, vp, vp, vp, C.POINTER(thermo_options), C.POINTER(vp)]
        L.thermo_set_density.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double]
        L.thermo_update_density.argtypes = [vp, vp, C.c_double, C.c_double, C.c_double]
        L.thermo_setup_precond.argtypes = [vp]
        L.thermo_solve.argtypes = [vp, vp, vp, C.c_double, C.POINTER(thermo_solve_info)]
        L.thermo_sensitivity.argtypes = [vp, vp, vp]
        L.thermo_compliance.argtypes = [vp, vp, dp]
        L.thermo_last_error.argtypes = [vp]
        L.thermo_last_error.restype = C.c_char_p
        L.thermo_destroy.argtypes = [vp]
        L.thermo_destroy.restype = None
        L.thermo_apply.argtypes = [vp, i, vp, vp]
        L.thermo_vcycle.argtypes = [vp, vp, vp]
        L.thermo_load_vector.argtypes = [vp, vp]
        L.thermo_hierarchy.argtypes = [vp, ip, ip, ip, C.POINTER(C.c_longlong)]
        L.thermo_export_level.argtypes = [vp, i, i, vp, C.c_longlong]
        L.thermo_filter.argtypes = [vp, vp, vp, C.c_double, i]
        L.thermo_oc_update.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, C.c_double, dp]
        L.thermo_launch_count.argtypes = []
        L.thermo_launch_count.restype = C.c_longlong
        L.thermo_bench_kernel.argtypes = [vp, i, i, dp, dp]
        L.thermo_apply_dot.argtypes = [vp, vp, vp, dp]
        L.thermo_kernel_timers.argtypes = [vp, i]
        L.thermo_dot_noalloc.argtypes = [vp, vp, C.c_longlong, vp, vp, C.c_char_p, i]
        L.thermo_residual_history.argtypes = [vp, C.POINTER(C.c_double), i]
        L.thermo_residual_history.restype = C.c_int
        L.thermo_kernel_time.argtypes = [vp, i, dp, C.POINTER(C.c_longlong), dp, dp]
        L.thermo_set_stage_wait.argtypes = [vp, C.c_longlong]
        L.thermo_dense_spd_inverse.argtypes = [i, vp, vp, vp, ip, C.c_char_p, i]
        d_ = C.c_double
        L.thermo_tpfa_conductivity.argtypes = [C.c_longlong, vp, d_, d_, d_, vp, vp]
        L.thermo_tpfa_apply.argtypes = [ip, dp, vp, vp, vp, vp, vp]
        L.thermo_tpfa_rhs.argtypes = [ip, dp, vp, d_, d_, vp, vp, d_, vp, vp]
        L.thermo_tpfa_sensitivity.argtypes = [ip, dp, vp, d_, d_, d_, d_, vp, vp, d_, vp, vp, vp, vp]
        for n in EXPORTED:
            if n not in ("thermo_last_error", "thermo_destroy", "thermo_launch_count"):
                getattr(L, n).restype = C.c_int
        _lib_handle = L
    return _lib_handle


def default_options(grid) -> thermo_options:
    o = thermo_options()
    g = (C.c_int * 3)(*grid)
    st = lib().thermo_default_options(g, C.byref(o))
    if st != OK:
        raise ThermoError(st, f"no default hierarchy for grid {tuple(grid)}")
    return o


def options(grid, **opts) -> thermo_options:
    """thermo_default_options(grid) with keyword overrides (nvec: list per
    level; group: list of sizes for levels 2..levels; other fields by name)."""
    o = default_options(grid)
    for k, v in opts.items():
        if k == "nvec":
            for j in range(MAX_LEVELS):
                o.nvec[j] = int(v[j]) if j < len(v) else 0
        elif k == "group":  # sizes for levels 2..levels
            o.group[0] = 0
            for j in range(1, MAX_LEVELS):
                o.group[j] = int(v[j - 1]) if j - 1 < len(v) else 0
        else:
            if not hasattr(o, k):
                raise AttributeError(f"unknown option {k}")
            setattr(o, k, v)
    return o


def plan_bytes(grid, has_dirichlet_value=False, **opts) -> int:
    """Device bytes a context for this grid and these options would allocate
    (thermo_plan_bytes: the allocation plan run without a GPU)."""
    o = options(grid, **opts)
    g = (C.c_int * 3)(*[int(v) for v in grid])
    n = C.c_longlong(0)
    st = lib().thermo_plan_bytes(g, C.byref(o), int(bool(has_dirichlet_value)), C.byref(n))
    if st != OK:
        raise ThermoError(st, f"thermo_plan_bytes rejected grid {tuple(grid)} / options")
    return int(n.value)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _dev(t, dtype):
    t = torch.as_tensor(t)
    if t.device.type != "cuda":
        t = t.to("cuda")
    return t.to(dtype).contiguous()


class Solver:
    """One libthermo context: Q1 heat operator + MMG-preconditioned CG.

    grid = (Nx, Ny, Nz) elements, h = element sizes, mask = uint8 node mask
    of Gamma_D, source = element heat source.  Keyword options override
    thermo_default_options: levels, block, group (list, per level >= 2),
    nvec (list), nu_fine, nu_coarse, omega, prec, pc, guess, max_iter,
    flexible, check_every.
    """

    def __init__(self, grid, h, mask, source, dirichlet_value=None, stream=None, **opts):
        self.grid = tuple(int(v) for v in grid)
        o = options(self.grid, **opts)
        self.options = o
        self.nnode = (self.grid[0] + 1) * (self.grid[1] + 1) * (self.grid[2] + 1)
        self.nelem = self.grid[0] * self.grid[1] * self.grid[2]
        mask = _dev(mask, torch.uint8)
        source = _dev(source, torch.float64)
        dval = None if dirichlet_value is None else _dev(dirichlet_value, torch.float64)
        if mask.numel() != self.nnode or source.numel() != self.nelem:
            raise ValueError("mask / source sizes do not match the grid")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._x = None
        ctx = C.c_void_p()
        g = (C.c_int * 3)(*self.grid)
        hh = (C.c_double * 3)(*[float(v) for v in h])
        st = lib().thermo_create(g, hh, _ptr(mask), _ptr(dval), _ptr(source),
                                 C.c_void_p(self.stream.cuda_stream), C.byref(o), C.byref(ctx))
        # the context keeps its own copies: the inputs are not retained
        self.stream.synchronize()
        del mask, source, dval
        self.ctx = ctx
        if st != OK:
            msg = self.last_error()
            self.close()
            raise ThermoError(st, msg)

    # -- helpers
    def last_error(self):
        if not self.ctx:
            return "no context"
        return lib().thermo_last_error(self.ctx).decode()

    def _check(self, st):
        if st != OK:
            raise ThermoError(st, self.last_error())
        return st

    def close(self):
        if getattr(self, "ctx", None):
            lib().thermo_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C ABI, same names
    def _design(self, x):
        return _dev(x, torch.float32 if self.options.density_fp32 else torch.float64)

    def set_density(self, x, p, kmin, kmax):
        self._x = self._design(x)
        return self._check(lib().thermo_set_density(self.ctx, _ptr(self._x), float(p), float(kmin), float(kmax)))

    def update_density(self, x, p, kmin, kmax):
        """thermo_update_density: new design, the current preconditioner kept."""
        self._x = self._design(x)
        return self._check(lib().thermo_update_density(self.ctx, _ptr(self._x), float(p), float(kmin), float(kmax)))

    def setup_precond(self):
        return self._check(lib().thermo_setup_precond(self.ctx))

    def solve(self, rhs=None, u=None, tol=1e-8, check=True):
        """Returns (u, info dict).  ``u`` is the initial guess for GIVEN /
        WARM_COARSE guesses and is overwritten with the solution."""
        if u is None:
            u = torch.zeros(self.nnode, dtype=torch.float64, device="cuda")
        r = None if rhs is None else _dev(rhs, torch.float64)
        info = thermo_solve_info()
        st = lib().thermo_solve(self.ctx, _ptr(r), _ptr(u), float(tol), C.byref(info))
        d = info.asdict()
        d["status_name"] = STATUS_NAMES.get(st, st)
        if check and st not in (OK,):
            raise ThermoError(st, self.last_error())
        return u, d

    def sensitivity(self, u, out=None):
        dc = out if out is not None else torch.empty(self.nelem, dtype=torch.float64, device="cuda")
        self._check(lib().thermo_sensitivity(self.ctx, _ptr(u), _ptr(dc)))
        return dc

    def compliance(self, u):
        c = C.c_double()
        self._check(lib().thermo_compliance(self.ctx, _ptr(u), C.byref(c)))
        return c.value

    def apply(self, u, precision=FP64):
        u = _dev(u, torch.float64)
        y = torch.empty_like(u)
        self._check(lib().thermo_apply(self.ctx, int(precision), _ptr(u), _ptr(y)))
        return y

    def apply_dot(self, p):
        """(q, p.q) with the fused FP64 kernel of the CG loop (p must vanish on Gamma_D)."""
        p = _dev(p, torch.float64)
        q = torch.empty_like(p)
        d = C.c_double()
        self._check(lib().thermo_apply_dot(self.ctx, _ptr(p), _ptr(q), C.byref(d)))
        return q, d.value

    def set_stage_wait(self, cycles=0):
        """Stage wait limit (clock64 cycles) of the TMA-staged fine kernels; 0 = default."""
        return self._check(lib().thermo_set_stage_wait(self.ctx, int(cycles)))

    def residual_history(self):
        """Relative recursive residuals of the last solve, one per convergence check."""
        n = lib().thermo_residual_history(self.ctx, None, 0)
        buf = (C.c_double * max(n, 1))()
        lib().thermo_residual_history(self.ctx, buf, n)
        return list(buf[:n])

    def kernel_timers(self, enable=True):
        """Start (zeroing the totals) or stop the per-kernel-class event timers of solve()."""
        self._check(lib().thermo_kernel_timers(self.ctx, 1 if enable else 0))

    def kernel_time(self, kclass):
        """(ms, launches, bytes, flops) summed over the timed launches of one class."""
        ms, b, f = C.c_double(), C.c_double(), C.c_double()
        n = C.c_longlong()
        self._check(lib().thermo_kernel_time(self.ctx, int(kclass), C.byref(ms), C.byref(n), C.byref(b), C.byref(f)))
        return ms.value, n.value, b.value, f.value

    def vcycle(self, r):
        r = _dev(r, torch.float64)
        z = torch.empty_like(r)
        self._check(lib().thermo_vcycle(self.ctx, _ptr(r), _ptr(z)))
        return z

    def load_vector(self):
        f = torch.empty(self.nnode, dtype=torch.float64, device="cuda")
        self._check(lib().thermo_load_vector(self.ctx, _ptr(f)))
        return f

    def hierarchy(self):
        n = C.c_int()
        cells = (C.c_int * (3 * MAX_LEVELS))()
        nvec = (C.c_int * MAX_LEVELS)()
        ndof = (C.c_longlong * MAX_LEVELS)()
        self._check(lib().thermo_hierarchy(self.ctx, C.byref(n), cells, nvec, ndof))
        return [dict(cells=tuple(cells[3 * l:3 * l + 3]), nvec=nvec[l], ndof=ndof[l]) for l in range(n.value)]

    def export_level(self, level, what, count):
        out = torch.empty(int(count), dtype=torch.float64, device="cuda")
        self._check(lib().thermo_export_level(self.ctx, int(level), int(what), _ptr(out), int(count)))
        return out

    def filter(self, x, rmin, transpose=False):
        x = _dev(x, torch.float64)
        y = torch.empty_like(x)
        self._check(lib().thermo_filter(self.ctx, _ptr(x), _ptr(y), float(rmin), int(bool(transpose))))
        return y

    def bench_kernel(self, which, reps=20):
        ms, by = C.c_double(), C.c_double()
        self._check(lib().thermo_bench_kernel(self.ctx, int(which), int(reps), C.byref(ms), C.byref(by)))
        return ms.value, by.value

    def oc_update(self, x, dc, dv, volfrac, move=0.2, rmin=1.5):
        ch = C.c_double()
        self._check(lib().thermo_oc_update(self.ctx, _ptr(x), _ptr(dc), _ptr(dv), float(volfrac),
                                           float(move), float(rmin), C.byref(ch)))
        return ch.value


def dot_noalloc(x, y, out):
    """out[0] = x . y through thermo_dot_noalloc (the library allocates nothing).
    x, y: contiguous CUDA float64 tensors of equal length; out: a CUDA float64
    tensor with at least one element, written on the current stream.  Only
    pointers are passed: nothing is converted or copied here."""
    for t in (x, y, out):
        if t.device.type != "cuda" or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError("dot_noalloc needs contiguous CUDA float64 tensors")
    if x.numel() != y.numel() or out.numel() < 1:
        raise ValueError("dot_noalloc: x and y must have equal length and out at least one element")
    msg = C.create_string_buffer(256)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().thermo_dot_noalloc(_ptr(x), _ptr(y), x.numel(), _ptr(out), st, msg, 256)
    if rc != OK:
        raise ThermoError(rc, msg.value.decode())
    return out


def dense_spd_inverse(A):
    """(A^-1, status, pivot, message) through thermo_dense_spd_inverse: the
    blocked FP64 Cholesky + inverse of the coarsest-level solve applied to a
    caller's dense matrix (CUDA float64 tensor, n x n, contiguous)."""
    if A.device.type != "cuda" or A.dtype != torch.float64 or A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("dense_spd_inverse needs a square CUDA float64 tensor")
    A = A.contiguous()
    X = torch.empty_like(A)
    piv = C.c_int(-1)
    msg = C.create_string_buffer(256)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().thermo_dense_spd_inverse(int(A.shape[0]), _ptr(A), _ptr(X), st, C.byref(piv), msg, 256)
    return X, rc, piv.value, msg.value.decode()


def resample(grid_c, v, grid_f, kind):
    """thermo_resample: carry a field from grid_c to grid_f = r * grid_c (kind 0:
    element field, piecewise constant; 1: element field, trilinear between cell
    centres; 2: nodal field, the coarse Q1 function at the fine nodes)."""
    v = _dev(v, torch.float64)
    e = 1 if kind == 2 else 0
    n = (int(grid_f[0]) + e) * (int(grid_f[1]) + e) * (int(grid_f[2]) + e)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    gc = (C.c_int * 3)(*[int(g) for g in grid_c])
    gf = (C.c_int * 3)(*[int(g) for g in grid_f])
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib().thermo_resample(gc, _ptr(v), gf, _ptr(out), int(kind), st)
    if rc != OK:
        raise ThermoError(rc, f"thermo_resample rejected {tuple(grid_c)} -> {tuple(grid_f)} kind {kind}")
    return out


class Tpfa:
    """The paper's cell-centred TPFA operator (thermo_tpfa_*): conductivity,
    A t, the right-hand side with the source f0 (1 - x^p) and the
    mean-temperature adjoint sensitivity, on device arrays in natural cell
    order.  dirichlet_faces: uint8 per cell, bit 2 axis + side."""

    def __init__(self, grid, h, dirichlet_faces):
        self.grid = tuple(int(v) for v in grid)
        self.h = tuple(float(v) for v in h)
        self.M = self.grid[0] * self.grid[1] * self.grid[2]
        self.dface = _dev(dirichlet_faces, torch.uint8)
        if self.dface.numel() != self.M:
            raise ValueError("dirichlet_faces must have one byte per cell")
        self._g = (C.c_int * 3)(*self.grid)
        self._h = (C.c_double * 3)(*self.h)

    def _st(self):
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)

    def _check(self, rc, what):
        if rc != OK:
            raise ThermoError(rc, f"{what} rejected its arguments")

    def conductivity(self, x, p, kmin, kmax):
        x = _dev(x, torch.float64)
        k = torch.empty_like(x)
        self._check(lib().thermo_tpfa_conductivity(self.M, _ptr(x), float(p), float(kmin), float(kmax), _ptr(k),
                                                   self._st()), "thermo_tpfa_conductivity")
        return k

    def apply(self, kappa, t):
        y = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self._check(lib().thermo_tpfa_apply(self._g, self._h, _ptr(_dev(kappa, torch.float64)), _ptr(self.dface),
                                            _ptr(_dev(t, torch.float64)), _ptr(y), self._st()), "thermo_tpfa_apply")
        return y

    def rhs(self, x, p, f0, kappa, TD):
        b = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self._check(lib().thermo_tpfa_rhs(self._g, self._h, _ptr(_dev(x, torch.float64)), float(p), float(f0),
                                          _ptr(_dev(kappa, torch.float64)), _ptr(self.dface), float(TD), _ptr(b),
                                          self._st()), "thermo_tpfa_rhs")
        return b

    def sensitivity(self, x, p, kmin, kmax, f0, kappa, TD, t, u):
        dc = torch.empty(self.M, dtype=torch.float64, device="cuda")
        self._check(lib().thermo_tpfa_sensitivity(self._g, self._h, _ptr(_dev(x, torch.float64)), float(p),
                                                  float(kmin), float(kmax), float(f0),
                                                  _ptr(_dev(kappa, torch.float64)), _ptr(self.dface), float(TD),
                                                  _ptr(_dev(t, torch.float64)), _ptr(_dev(u, torch.float64)),
                                                  _ptr(dc), self._st()), "thermo_tpfa_sensitivity")
        return dc


def launch_count() -> int:
    """Kernel launches issued by libthermo so far in this process."""
    return int(lib().thermo_launch_count())
