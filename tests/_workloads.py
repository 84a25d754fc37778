"""Workload variants built from the generator's meshes, shared by CPU and GPU tests."""
import dataclasses

import numpy as np

from paper_2403_09198_gb300 import inputs


def subset_blocks(w, keep):
    """The workload restricted to the blocks where ``keep`` is True (diagonal
    blocks always kept), with their S values and pairs in the same order."""
    keep = np.asarray(keep) | w.is_diag_block()
    ks = np.flatnonzero(keep)
    so, pi = w.s_offsets(), w.pair_indptr.astype(np.int64)
    rows = np.repeat(np.arange(w.n_cells), np.diff(w.block_indptr))
    block_indptr = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=w.n_cells))])
    pair_indptr = np.concatenate([[0], np.cumsum(np.diff(pi)[keep])])
    return dataclasses.replace(
        w, block_indptr=block_indptr.astype(np.int32), block_indices=w.block_indices[keep].copy(),
        pair_indptr=pair_indptr.astype(np.int32),
        S=np.concatenate([w.S[so[k]:so[k + 1]] for k in ks]),
        U=np.concatenate([w.U[pi[k]:pi[k + 1]] for k in ks]),
        V=np.concatenate([w.V[pi[k]:pi[k + 1]] for k in ks]))


def nonsymmetric(Lx=7, Ly=6, N=12, seed=21):
    """A block pattern that is not symmetric: every row keeps its diagonal and
    its lower neighbours, and one interior cell keeps its whole row (5 blocks in
    the widest row, 4 in the widest column)."""
    w0 = inputs.make_workload(Lx, Ly, N=N, w=2, r_diag=2, r_off=1, seed=seed)
    rows = np.repeat(np.arange(w0.n_cells), np.diff(w0.block_indptr))
    c = (Ly // 2) * Lx + Lx // 2
    return subset_blocks(w0, (w0.block_indices < rows) | (rows == c))
