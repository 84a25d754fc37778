"""Helpers shared by the GPU parity tests."""
import functools

import numpy as np

import oracle
from paper_2403_09198_gb300 import inputs

# Tolerance of the FP64 path against the FP64 oracle (relative).
TOL64 = 1e-12

# Small workloads the oracle finishes in seconds; together they cover several
# tiles and ragged tails, one cell, 1 x L strips, N = 1, no pairs, the paper's
# physical pair counts (9 per diagonal block, 2 per neighbour block), the
# band +-4 / 3-pair family of the N = 200 workload, two patterns outside the
# paper's family (a shared pattern, random patterns) that take the generic
# table-driven kernels, and pair counts that differ from block to block.
SMALL = {
    "grid16_N10": dict(Lx=16, N=10, w=2, r_diag=2, r_off=1, seed=0),
    "ragged5x3": dict(Lx=5, Ly=3, N=4, w=1, r_diag=2, r_off=1, seed=1),
    "one_cell": dict(Lx=1, Ly=1, N=3, w=1, r_diag=1, r_off=0, seed=2),
    "strip1x40": dict(Lx=1, Ly=40, N=2, w=1, r_diag=2, r_off=1, seed=3),
    "N1": dict(Lx=9, Ly=7, N=1, w=0, r_diag=2, r_off=1, seed=4),
    "no_pairs": dict(Lx=6, Ly=6, N=5, w=2, r_diag=0, r_off=0, seed=5),
    "pairs9_2": dict(Lx=6, Ly=5, N=8, w=2, r_diag=9, r_off=2, seed=6),
    "same_pattern": dict(Lx=8, Ly=4, N=6, w=2, r_diag=2, r_off=1, seed=7, same_pattern=True),
    "band4_r3": dict(Lx=33, Ly=2, N=12, w=4, r_diag=3, r_off=1, seed=8),
    "random_pattern": dict(Lx=7, Ly=6, N=9, r_diag=2, r_off=1, seed=10, random_density=0.3),
    # per-block pair counts: 1 + 2 per face on diagonal blocks (9 / 7 / 5), 2 per
    # neighbour block; and counts drawn from 0..3 per block, zero-pair blocks included
    "pairs_faces": dict(Lx=6, Ly=5, N=8, w=2, r_diag=1, r_off=2, pairs_per_face=2, seed=11),
    "pairs_random": dict(Lx=9, Ly=5, N=7, w=2, r_diag=0, r_off=0, random_pair_max=3, seed=12),
}


def workload(name):
    return inputs.make_workload(**SMALL[name])


@functools.lru_cache(maxsize=4)
def full(name):
    """A full-size named workload, generated once per test session."""
    return inputs.named_workload(name)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel_err(got, ref):
    """Largest element error, each scaled by max(|ref_i|, 1e-3 ||ref||_inf),
    and the norm-wise relative error; the larger of the two."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    if ref.size == 0:
        return 0.0
    scale = np.maximum(np.abs(ref), 1e-3 * max(np.abs(ref).max(), 1e-300))
    elem = float(np.max(np.abs(got - ref) / scale))
    norm = float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))
    return max(elem, norm)


def sol_err(got, ref):
    """Norm-wise relative difference, used for solver outputs."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300))


def to_component_major(v, nc, b):
    return np.ascontiguousarray(np.asarray(v).reshape(nc, b).T).ravel()


def from_component_major(v, nc, b):
    return np.ascontiguousarray(np.asarray(v).reshape(b, nc).T).ravel()


def oracle_jac(w, S=None, U=None, V=None):
    return oracle.Jacobian.from_workload(w, S=S, U=U, V=V)
