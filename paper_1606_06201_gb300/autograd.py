"""Differentiable displacement and compliance: torch.autograd.Function wrappers of the MGCG solve.

For u(x) with K(x) u = f (Eq. (to)) and a scalar loss L(u), the adjoint system K(x) lam = dL/du
is solved by a second MGCG solve (same hierarchy, rebuilt when the solver was reused in between)
and dL/dx_e = -lam_e^T K0 u_e is formed by one element kernel.  For the compliance c = f^T u the
adjoint is lam = u, so dc/dx_e = -u_e^T K0 u_e needs no second solve (the energy term of KKT3,
Sec. 2).  Everything runs in the CUDA library; this module only wires it into autograd.
"""
import torch

from . import topo


class _Displacement(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, f, solver, tol, adjoint_tol):
        solver.set_density(x.detach().contiguous())
        u, info = solver.solve(f.detach().contiguous(), tol=tol)
        ctx.solver, ctx.tol = solver, adjoint_tol
        ctx.save_for_backward(x.detach(), u)
        ctx.info = info
        return u

    @staticmethod
    def backward(ctx, grad_u):
        x, u = ctx.saved_tensors
        s = ctx.solver
        # the hierarchy is recomputed rather than kept, so the solver may serve other calls
        s.set_density(x.contiguous())
        lam, _ = s.solve(grad_u.contiguous(), tol=ctx.tol)
        g = s.grad_x(lam, u)
        return g, None, None, None, None


class _Compliance(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, f, solver, tol):
        solver.set_density(x.detach().contiguous())
        u, info = solver.solve(f.detach().contiguous(), tol=tol)
        c = torch.as_tensor(float(solver.compliance(f.detach().contiguous(), u)[0]),
                            dtype=torch.float64, device=x.device)
        ctx.solver = solver
        ctx.save_for_backward(u)
        ctx.info = info
        return c

    @staticmethod
    def backward(ctx, grad_c):
        (u,) = ctx.saved_tensors
        g = ctx.solver.grad_x(u, u)
        return grad_c * g, None, None, None


def displacement(x, f, solver, tol=1e-10, adjoint_tol=None):
    """u(x) solving K(x) u = f; differentiable in x through the adjoint MGCG."""
    return _Displacement.apply(x, f, solver, tol, tol if adjoint_tol is None else adjoint_tol)


def compliance(x, f, solver, tol=1e-10):
    """c(x) = f^T u(x); differentiable in x (dc/dx_e = -u_e^T K0 u_e)."""
    return _Compliance.apply(x, f, solver, tol)


__all__ = ["displacement", "compliance", "topo"]
