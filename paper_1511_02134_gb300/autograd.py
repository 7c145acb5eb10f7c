"""torch.autograd wrapper: the Stokes solve as a differentiable map of the
nodal body force.

forward(f) -> (u, p): right-hand side from f and the mesh's Dirichlet data
(Sec. 2.1 forms), then the multigrid solve (hhg_set_rhs + hhg_solve).
backward(dJ/du, dJ/dp) -> dJ/df: K is symmetric (Sec. 3), so the adjoint
system K lambda = (dJ/du, dJ/dp) is solved by the same multigrid and the
gradient is R^T lambda with R f = (M f, sum_d G_d f_d) (hhg_adjoint_gradient).
No activations are stored: the operator is matrix-free and linear.  Needs a
mesh with an outflow face (non-singular K).
"""
from __future__ import annotations

import torch

from . import MODE_FP64


class StokesSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f, mesh, u_dirichlet=None, tol=1e-10, max_cycles=60, mode=MODE_FP64):
        f = f.detach().contiguous()
        if f.is_cuda:
            torch.cuda.current_stream(f.device).synchronize()
        mesh.set_rhs(f, u_dirichlet)
        u = torch.empty_like(f)
        p = torch.empty(f.shape[0], dtype=f.dtype, device=f.device)
        mesh.solve(tol=tol, max_cycles=max_cycles, mode=mode, u_out=u, p_out=p)
        ctx.mesh, ctx.tol, ctx.max_cycles, ctx.mode = mesh, tol, max_cycles, mode
        return u, p

    @staticmethod
    def backward(ctx, grad_u, grad_p):
        gu = grad_u.contiguous() if grad_u is not None else None
        gp = grad_p.contiguous() if grad_p is not None else None
        ref = gu if gu is not None else gp
        if ref.is_cuda:
            torch.cuda.current_stream(ref.device).synchronize()
        out = torch.empty((ref.shape[0], 3), dtype=torch.float64, device=ref.device)
        ctx.mesh.adjoint_gradient(ju=gu, jp=gp, tol=ctx.tol, max_cycles=ctx.max_cycles, mode=ctx.mode, out=out)
        return out, None, None, None, None, None


def stokes_solve(f, mesh, u_dirichlet=None, tol=1e-10, max_cycles=60, mode=MODE_FP64):
    """(u, p) = solution for nodal body force f (n, 3) float64; differentiable in f."""
    return StokesSolve.apply(f, mesh, u_dirichlet, tol, max_cycles, mode)
