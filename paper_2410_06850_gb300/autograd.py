"""torch.autograd wrappers around the C ABI.

ComplianceFn: c(x) = f^T u(x) with A(x) u = f (Sec. 2.3).  forward() sets the
design, builds the preconditioner and solves; backward() returns
grad_c * dc/dx with the adjoint sensitivity kernel (the operator is
self-adjoint and the load does not depend on x, so the adjoint is the state:
dc/dx_e = -p x_e^(p-1) (kmax - kmin) u_e^T K0 u_e).

FilterFn: the hat-weight density filter (SIMP harness, not in the paper); it
is linear, so backward applies its transpose.
"""
from __future__ import annotations

import torch


class ComplianceFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, solver, p=3.0, kmin=1e-3, kmax=1.0, tol=1e-8, u0=None):
        solver.set_density(x.detach(), p, kmin, kmax)
        solver.setup_precond()
        u, info = solver.solve(u=None if u0 is None else u0.detach().clone(), tol=tol)
        c = solver.compliance(u)
        ctx.solver = solver
        ctx.params = (p, kmin, kmax)
        ctx.x = x.detach()
        ctx.save_for_backward(u)
        solver.last_info = info
        solver.last_u = u
        return torch.tensor(c, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, grad_c):
        (u,) = ctx.saved_tensors
        s = ctx.solver
        if s._x is None or s._x.data_ptr() != ctx.x.data_ptr():
            s.set_density(ctx.x, *ctx.params)
        dc = s.sensitivity(u)
        return grad_c * dc, None, None, None, None, None, None


class FilterFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, solver, rmin=1.5):
        ctx.solver = solver
        ctx.rmin = rmin
        return solver.filter(x.detach(), rmin, transpose=False)

    @staticmethod
    def backward(ctx, g):
        return ctx.solver.filter(g.contiguous(), ctx.rmin, transpose=True), None, None


def compliance(x, solver, p=3.0, kmin=1e-3, kmax=1.0, tol=1e-8, u0=None):
    return ComplianceFn.apply(x, solver, p, kmin, kmax, tol, u0)


def density_filter(x, solver, rmin=1.5):
    return FilterFn.apply(x, solver, rmin)
