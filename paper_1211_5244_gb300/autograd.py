"""torch.autograd wrapper of the solve with the library's adjoint.

    V, E = hartree(rho, plan)

V = K rho (Eq. 2) and E = 1/2 h^3 <rho, V>. The backward pass calls
ps_solve_vjp: K is even, so the operator is symmetric and the
vector-Jacobian product through V is the same convolution applied to the
incoming gradient; the energy's gradient is h^3 V from the forward result.
Both run in the library's kernels.
"""
from __future__ import annotations

import torch


class HartreeSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, plan):
        ctx.set_materialize_grads(False)  # an unused output gets None, not a zero tensor
        V, E = plan.solve(rho.contiguous())
        ctx.plan = plan
        ctx.save_for_backward(V)
        return V, E

    @staticmethod
    def backward(ctx, gV, gE):
        (V,) = ctx.saved_tensors
        plan = ctx.plan
        vbar = gV.contiguous() if gV is not None else None
        gE64 = gE.detach().to(torch.float64).reshape(()) if gE is not None else None
        if vbar is None and gE64 is None:
            return None, None
        grad = plan.solve_vjp(vbar=vbar, V=V if gE64 is not None else None, gE=gE64)
        return grad, None


def hartree(rho, plan):
    """(V, E) with gradients through the library's adjoint."""
    return HartreeSolve.apply(rho, plan)
