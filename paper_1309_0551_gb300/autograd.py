"""torch.autograd.Function around dslash_force: the pseudofermion action
S = Re chi^dag (m^2 - D_eo D_oe) chi and its backward (fermion force).

Argument marshalling only: the forward calls dslash_force for S, the backward calls it
again for dS/dU and dS/dchi, recomputing D_oe chi instead of keeping it from the forward.
Gradients follow PyTorch's convention for real functions of complex tensors
(dS/dRe + i dS/dIm), which is the library's G = 2 Z^dag and 2 M chi.
"""
from __future__ import annotations

import torch

from . import Context, lq_gauge_pack, dslash_force, PREC


class DslashAction(torch.autograd.Function):
    """S = DslashAction.apply(U, chi, mass, ctx, dims).

    U: complex128 CUDA tensor (4, V, 3, 3) (canonical gauge layout); chi: complex128 or
    complex64 CUDA tensor (Vh, 3) on the even sites -- its dtype selects FP64 or FP32
    arithmetic (the links are packed to the same precision on each call)."""

    @staticmethod
    def forward(fctx, U, chi, mass, ctx: Context, dims):
        prec = "f64" if chi.dtype == torch.complex128 else "f32"
        g = lq_gauge_pack(ctx, dims, U.detach().contiguous(), prec, 18)
        S = dslash_force(ctx, g, mass, chi.detach().contiguous(), want_S=True)
        fctx.save_for_backward(U, chi)
        fctx.mass, fctx.ctx, fctx.dims, fctx.prec = mass, ctx, dims, prec
        return torch.tensor(S, dtype=torch.float64 if prec == "f64" else torch.float32, device=chi.device)

    @staticmethod
    def backward(fctx, grad_S):
        U, chi = fctx.saved_tensors
        ctx = fctx.ctx
        g = lq_gauge_pack(ctx, fctx.dims, U.detach().contiguous(), fctx.prec, 18)
        ctype = torch.complex128 if fctx.prec == "f64" else torch.complex64
        dU = torch.empty(U.shape, dtype=ctype, device=U.device) if fctx.needs_input_grad[0] else None
        dchi = torch.empty_like(chi) if fctx.needs_input_grad[1] else None
        dslash_force(ctx, g, fctx.mass, chi.detach().contiguous(), dSdU=dU, dSdchi=dchi)
        gU = None if dU is None else (dU * grad_S).to(U.dtype)
        gchi = None if dchi is None else dchi * grad_S
        return gU, gchi, None, None, None


def force_ta(ctx: Context, U, chi, mass: float, dims):
    """The projected force F = TA(U G^dag), canonical (4, V, 3, 3), in chi's precision."""
    prec = "f64" if chi.dtype == torch.complex128 else "f32"
    g = lq_gauge_pack(ctx, dims, U.contiguous(), PREC[prec], 18)
    F = torch.empty(U.shape, dtype=chi.dtype, device=U.device)
    dslash_force(ctx, g, mass, chi.contiguous(), force_TA=F)
    return F
