"""Gradient of the implicit solve x = J^-1 b (test infrastructure only).

For the loss L = 0.5 ||W x||^2 with W diagonal: dL/dx = W^2 x, the adjoint
lambda solves J^T lambda = W^2 x, and then dL/db = lambda and dL/dJ = -lambda x^T,
restricted to the stored parameters: the S pattern entries and the rank-one
factors (dL/du = -(v . x_j) lambda_i, dL/dv = -(u . lambda_i) x_j).
"""
from __future__ import annotations

import numpy as np

from .gmres import gmres
from .native import Jacobian, bj_setup, grad


def adjoint(J: Jacobian, b, Wdiag, rtol: float = 1e-14, restart: int = 30,
            max_iters: int = 1000):
    """Return dict(x, lam, loss, gb, gS, gU, gV, info_fwd, info_adj)."""
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    Wdiag = np.ascontiguousarray(Wdiag, dtype=np.float64).ravel()
    F = bj_setup(J)
    x, info_f = gmres(J, b, restart=restart, rtol=rtol, max_iters=max_iters, factors=F)
    loss = 0.5 * float(np.dot(Wdiag * x, Wdiag * x))
    gx = Wdiag * Wdiag * x
    lam, info_a = gmres(J, gx, restart=restart, rtol=rtol, max_iters=max_iters, trans=True,
                        factors=F)
    gS, gU, gV = grad(J, lam, x)
    return dict(x=x, lam=lam, loss=loss, gb=lam, gS=gS, gU=gU, gV=gV,
                info_fwd=info_f, info_adj=info_a)
