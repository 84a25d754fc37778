"""Textbook restarted, right-preconditioned GMRES(m) in FP64 (test infrastructure only).

Saad & Schultz's GMRES with the right preconditioning of Section 6: solve
(A M) y = b, x = M y.  Each cycle starts from the true residual r = b - A x,
builds an orthonormal Krylov basis V by modified Gram-Schmidt, reduces the
Hessenberg matrix H to triangular form by Givens rotations, and stops when the
rotated residual |g_{j+1}| / ||b|| reaches ``rtol``; the correction is
x += M (V_k y_k) with R y_k = g.  At every restart and at the end the true
residual ||b - A x|| / ||b|| is recomputed and convergence is declared only on
it.  A happy breakdown is taken when h_{j+1,j} <= 1e-14 ||w||, ||w|| the norm of
A M v_j before orthogonalisation.

Left preconditioning (Section 6, Eq. left_precond_system, (M A) x = M b): a cycle
starts from z = M (b - A x), the Arnoldi operator is M A, the correction is
x += V_k y_k, and a cycle stops when |g_{j+1}| has fallen below ||z|| times the
factor rtol ||b|| / ||b - A x|| that the true residual still needs; the
history holds |g_{j+1}| / ||z|| times the cycle's starting true relative
residual.  Convergence is again declared only on the recomputed true residual.
"""
from __future__ import annotations

import math
from typing import Callable

import numpy as np

from .native import Jacobian, bj_apply, bj_setup, matvec


def _gmres_core(A: Callable, M: Callable, b: np.ndarray, m: int, rtol: float,
                max_iters: int, x0=None, left: bool = False):
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = float(np.linalg.norm(b))
    info = dict(iterations=0, restarts=0, history=[], true_rel=0.0, converged=True,
                breakdown=False)
    if bnorm == 0.0:
        x[:] = 0.0
        return x, info
    its = 0
    while True:
        r = b - A(x)
        beta = float(np.linalg.norm(r))
        info["true_rel"] = beta / bnorm
        if beta / bnorm <= rtol:
            info["converged"] = True
            break
        if its >= max_iters:
            info["converged"] = False
            break
        Vb = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        if left:
            z = M(r)
            g0 = float(np.linalg.norm(z))
            Vb[0] = z / g0
            stop = g0 * (rtol * bnorm / beta)
            scale = beta / (g0 * bnorm)
        else:
            g0 = beta
            Vb[0] = r / beta
            stop = rtol * bnorm
            scale = 1.0 / bnorm
        g[0] = g0
        k = 0
        for j in range(m):
            w = M(A(Vb[j])) if left else A(M(Vb[j]))
            w0 = float(np.linalg.norm(w))
            for i in range(j + 1):                  # modified Gram-Schmidt
                H[i, j] = float(np.dot(w, Vb[i]))
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            for i in range(j):                      # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            hjj, hj1 = H[j, j], H[j + 1, j]
            denom = math.hypot(hjj, hj1)
            cs[j], sn[j] = hjj / denom, hj1 / denom
            H[j, j] = denom
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            k = j + 1
            info["history"].append(abs(g[j + 1]) * scale)
            happy = hj1 <= 1e-14 * w0
            if happy:
                info["breakdown"] = True
            if happy or abs(g[j + 1]) <= stop or its >= max_iters:
                break
            Vb[j + 1] = w / hj1
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):              # back substitution R y = g
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + (Vb[:k].T @ y if left else M(Vb[:k].T @ y))
        info["restarts"] += 1
    info["iterations"] = its
    return x, info


def gmres(J: Jacobian, b, restart: int = 30, rtol: float = 1e-10, max_iters: int = 1000,
          precond: str = "bj", trans: bool = False, x0=None, factors=None, left: bool = False):
    """Solve J x = b (or J^T x = b) with block-Jacobi right (``left``: left) preconditioning.

    Returns ``(x, info)``; ``info`` holds iterations, restarts, the per-iteration
    rotated residual history, the final true relative residual and ``converged``.
    """
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    if precond == "bj":
        F = bj_setup(J) if factors is None else factors

        def M(v):
            return bj_apply(F, v, trans=trans)
    elif precond == "none":
        def M(v):
            return v
    else:
        raise ValueError("precond must be 'bj' or 'none'")

    def A(v):
        return matvec(J, v, trans=trans)

    return _gmres_core(A, M, b, restart, rtol, max_iters, x0=x0, left=left)


def gmres_operator(A: Callable, M: Callable, b, restart: int, rtol: float,
                   max_iters: int = 1000, x0=None, left: bool = False):
    """The same textbook GMRES on caller-supplied operators (small dense tests)."""
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    return _gmres_core(A, M, b, restart, rtol, max_iters, x0=x0, left=left)
