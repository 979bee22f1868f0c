"""torch.autograd wrapper of K multigrid cycles (the hand-written adjoint).

    u_K = vcycles(b, coeffs, solver, K)

runs K cycles from u_0 = 0 with the solver's cycle (V(nu1, nu2), its
precision) and the omega-folded SPAI weights `coeffs` (a CPU float64 tensor
that may require grad); backward calls mg_vcycles_adjoint, which returns
dL/db on the GPU and dL/dcoeffs accumulated in FP64. All arithmetic runs in
the CUDA library; this module only moves tensors across the C ABI.
"""
from __future__ import annotations

import torch

from .binding import Solver


class _VCycles(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, coeffs, solver: Solver, K: int):
        c = tuple(float(x) for x in coeffs.detach().cpu().tolist())
        if c != tuple(solver.coeffs):
            solver.set_coeffs(c)
        u = solver.cycles(b, K)
        ctx.solver, ctx.K = solver, K
        ctx.save_for_backward(b, coeffs)
        return u

    @staticmethod
    def backward(ctx, grad_u):
        b, coeffs = ctx.saved_tensors
        solver = ctx.solver
        c = tuple(float(x) for x in coeffs.detach().cpu().tolist())
        if c != tuple(solver.coeffs):
            solver.set_coeffs(c)
        gb, gc = solver.vcycles_adjoint(b, grad_u.contiguous(), ctx.K)
        return gb, torch.as_tensor(gc, dtype=coeffs.dtype, device=coeffs.device), None, None


def vcycles(b, coeffs, solver: Solver, K: int):
    """u_K after K cycles from zero; differentiable w.r.t. b and coeffs."""
    return _VCycles.apply(b, coeffs, solver, K)
