"""torch.autograd.Function for <O>_inf = Tr(O rho_inf) through the C ABI (implicit differentiation,
Remark "Differentiating the steady state").

Forward: lindblad_setup + steady_state.  Backward: steady_state_adjoint, whose sensitivities gH, gL
satisfy dJ = Re<gH, dH> + sum_j Re<gL_j, dL_j>, which is exactly the gradient convention of torch for a
real output and complex inputs.  Marshalling only; every step runs in liblindblad.so.
"""
from __future__ import annotations

import torch

from . import lindblad as _B


class SteadyStateExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H, L, O, tol=1e-12):
        H = H.detach().contiguous()
        L = L.detach().contiguous()
        O = O.detach().contiguous()
        opts = _B.default_opts(tol=tol, max_restarts=100)
        h = _B.lindblad_setup(H, L, opts)
        rho, info, st = _B.steady_state(h, opts)
        if st != 0:
            _B.lindblad_destroy(h)
            raise _B.LindbladError(st, "steady_state")
        ctx.handle, ctx.opts = h, opts
        ctx.save_for_backward(rho, O)
        return (O * rho.transpose(0, 1)).sum().real   # Tr(O rho) without an n^3 product

    @staticmethod
    def backward(ctx, gJ):
        rho, O = ctx.saved_tensors
        h = ctx.handle
        _, gH, gL, info, st = _B.steady_state_adjoint(h, rho, O, ctx.opts)
        _B.lindblad_destroy(h)
        g = gJ.to(torch.float64)
        return gH * g, gL * g, None, None


def steady_state_expectation(H, L, O, tol=1e-12):
    """<O> in the steady state of (H, {L_j}); differentiable in H and L (complex128 CUDA tensors)."""
    return SteadyStateExpectation.apply(H, L, O, tol)
