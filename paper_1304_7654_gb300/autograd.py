"""torch.autograd.Function wrappers over the library's reverse-mode adjoint.

HBResidual: R = R_HB(U); backward(psi) = (dR/dU)^T psi (hb_adjoint_residual
with J_seed = 0).  HBLift: J = time-averaged lift; backward(g) = g dJ/dU
(hb_adjoint_residual with psi = 0, J_seed = g).  Both run only the
library's CUDA kernels; U must be a CUDA FP64 tensor in the context layout.
"""
from __future__ import annotations

import torch


class HBResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, hbctx):
        ctx.hbctx = hbctx
        ctx.save_for_backward(U)
        return hbctx.residual(U)

    @staticmethod
    def backward(ctx, gR):
        (U,) = ctx.saved_tensors
        r_adj, _ = ctx.hbctx.adjoint_residual(U, gR.contiguous(), 0.0)
        return r_adj, None


class HBLift(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, hbctx):
        ctx.hbctx = hbctx
        ctx.save_for_backward(U)
        _, J = hbctx.forces(U)
        return J.reshape(())

    @staticmethod
    def backward(ctx, gJ):
        (U,) = ctx.saved_tensors
        psi = torch.zeros_like(U)
        # the adjoint is linear in the seed: scale the unit-seed adjoint by gJ
        # on the device instead of reading gJ on the host (no stream sync)
        r_adj, _ = ctx.hbctx.adjoint_residual(U, psi, 1.0)
        return r_adj * gJ.to(r_adj.dtype), None


def residual(U, hbctx):
    return HBResidual.apply(U, hbctx)


def lift(U, hbctx):
    return HBLift.apply(U, hbctx)
