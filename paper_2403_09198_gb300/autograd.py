"""Differentiable implicit solve x = J^-1 b on the block r1-sparse Jacobian.

Forward: load the values, set up SMW block-Jacobi and run right-preconditioned
GMRES.  Backward: the adjoint lambda = J^-T g_x from GMRES on the transposed
operators (transposed matvec and transposed SMW block-Jacobi), then
g_b = lambda and the outer products g_S = -lambda x^T on the S pattern,
g_u = -(v . x_j) lambda_i, g_v = -(u . lambda_i) x_j, all in the CUDA library.
"""
from __future__ import annotations

import torch

from .binding import StsJacobian


class ImplicitSolve(torch.autograd.Function):
    """``x = ImplicitSolve.apply(b, S, U, V, jac, rtol, restart)``.

    ``jac`` is a :class:`StsJacobian` created with ``transpose=True`` on the same
    structure; its values are replaced by (S, U, V) in the forward pass.  One
    handle may serve several solves of one graph (for example unrolled
    pseudo-time steps): the backward pass reloads this solve's (S, U, V) and
    sets the preconditioner up again when the handle's values have changed
    since its forward pass.
    """

    @staticmethod
    def forward(ctx, b, S, U, V, jac: StsJacobian, rtol: float = 1e-10, restart: int = 30):
        S, U, V = S.detach(), U.detach(), V.detach()
        jac.update_values(S, U, V)
        jac.bjacobi_setup()
        x, info = jac.gmres(b.detach(), rtol=rtol, restart=restart)
        ctx.jac = jac
        ctx.rtol = rtol
        ctx.restart = restart
        ctx.version = jac.values_version
        ctx.save_for_backward(x, S, U, V)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, gx):
        x, S, U, V = ctx.saved_tensors
        jac: StsJacobian = ctx.jac
        if jac.values_version != ctx.version:
            # another solve (or a Newton step) has loaded other values since
            jac.update_values(S, U, V)
            jac.bjacobi_setup()
            ctx.version = jac.values_version
        lam, _ = jac.gmres(gx.contiguous(), rtol=ctx.rtol, restart=ctx.restart, trans=True)
        gS, gU, gV = jac.grad(lam, x)
        return lam, gS, gU, gV, None, None, None
