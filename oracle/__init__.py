"""Plain FP64 CPU oracle for the block r1-sparse Jacobian path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library and never imports it.

What it computes (each a plain definition, no blocking or reordering):

* ``matvec``          y = D x, D the dense block matrix D_ij = S_ij + sum u v^T
                       (Section 4.3, Section 5.1 BR1-BSR storage, Section 5.2).
* ``bj_setup/apply``  block-Jacobi M = blockdiag(D)^-1 by per-cell dense LU with
                       partial pivoting (Section 6).
* ``gmres``           textbook restarted GMRES(m) with modified Gram-Schmidt and
                       Givens rotations, right-preconditioned (Section 6, x = M y,
                       (A M) y = b) or, with ``left=True``, left-preconditioned
                       ((M A) x = M b).
* ``grad``/``adjoint`` gradients of L = 0.5 ||W x||^2 for x = J^-1 b through the
                       adjoint system J^T lambda = W^2 x.
* ``flux`` (module)    the HLL flux of a toy N-species flow model, its Jacobian
                       parts (Section 4.1, sparse part plus two rank-one pairs per
                       face), the first-order finite-volume residual (Section 3.3),
                       the BR1-BSR blocks of dR/dQ and a dense Newton iteration.

Parity status: every function above is pinned by the ``-m "not gpu"`` tests
(paper worked examples, library special cases, invariants, brute force, and
complex-step derivatives for ``flux``); planted mistakes trip those pins
(``tests/test_oracle_mutations.py``, ``tests/test_flux_pins.py``).
"""
from .native import (OracleSingular, BJFactors, Jacobian, bj_apply, bj_cells, bj_setup,
                     build, grad, matvec, matvec_rows, max_threads)
from .gmres import gmres
from .adjoint import adjoint

__all__ = ["OracleSingular", "BJFactors", "Jacobian", "bj_apply", "bj_cells", "bj_setup",
           "build", "grad", "matvec", "matvec_rows", "max_threads", "gmres", "adjoint"]
