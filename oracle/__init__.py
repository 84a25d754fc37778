"""Plain FP64 CPU oracle for the block r1-sparse Jacobian path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library and never imports it.

What it computes (each a plain definition, no blocking or reordering):

* ``matvec``          y = D x, D the dense block matrix D_ij = S_ij + sum u v^T
                       (Section 4.3, Section 5.1 BR1-BSR storage, Section 5.2).
* ``bj_setup/apply``  block-Jacobi M = blockdiag(D)^-1 by per-cell dense LU with
                       partial pivoting (Section 6).
* ``gmres``           textbook restarted right-preconditioned GMRES(m) with
                       modified Gram-Schmidt and Givens rotations (Section 6,
                       right preconditioning x = M y, (A M) y = b).
* ``grad``/``adjoint`` gradients of L = 0.5 ||W x||^2 for x = J^-1 b through the
                       adjoint system J^T lambda = W^2 x.

Parity status: every function above is pinned by the ``-m "not gpu"`` tests
(paper worked examples, library special cases, invariants, brute force).
"""
from .native import (OracleSingular, BJFactors, Jacobian, bj_apply, bj_cells, bj_setup,
                     build, grad, matvec, matvec_rows, max_threads)
from .gmres import gmres
from .adjoint import adjoint

__all__ = ["OracleSingular", "BJFactors", "Jacobian", "bj_apply", "bj_cells", "bj_setup",
           "build", "grad", "matvec", "matvec_rows", "max_threads", "gmres", "adjoint"]
