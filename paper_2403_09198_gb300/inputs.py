"""Seeded synthetic workloads shaped like the paper's structured-grid StS Jacobians.

This module builds problem *inputs* only: the mesh adjacency, the two intra-block
sparsity patterns, and random values drawn from a seeded numpy PCG64 stream.  It
holds none of the method's arithmetic (no products, solves or assembly), so the
CUDA path and the FP64 oracle can both consume its output without sharing code.

Layout of one workload (all arrays numpy, C-contiguous):

* Cells of an ``Lx x Ly`` structured quad grid, id ``iy*Lx + ix`` (Section 5.1:
  the BSR index arrays are fixed by the mesh adjacency).  ``block_indptr[nc+1]``
  and ``block_indices[nnzb]`` (int32) list, per block row, the cell itself and its
  up-to-four face neighbours ``i-Lx, i-1, i+1, i+Lx``, sorted ascending.  A
  boundary face adds no block ("zero-flux" reading of the boundary conditions).
* Block size ``b = N + 3``: N level densities, two momenta, one energy, in that
  order (Section 2.1 gives m = N_s + 3).
* Diagonal-block pattern (b x b CSR, row-major, ascending columns): level row p
  has the level band ``|p-q| <= w`` plus the three flow columns; the three flow
  rows are dense (Figures 2, 4 and 6 of Section 4).  nnz = (2w+1)N - w(w+1) + 3N + 3b.
* Off-diagonal-block pattern: level row p has the diagonal entry plus the three
  flow columns; flow rows dense (flux Jacobian pattern of Figure 2), nnz = 7N + 9.
  ``same_pattern=True`` reuses the diagonal pattern instead.
* S values: block order x pattern order, diagonal blocks hold nnz_d values, the
  others nnz_o.  Pairs: ``r_diag`` per diagonal block and ``r_off`` per
  off-diagonal block, pair order = block order (BR1-BSR ``pair_indptr`` of
  Section 5.1); ``U`` (column_data) and ``V`` (row_data) are ``[n_pairs][b]``.
* Per-block pair counts (Section 5.1 allows them to differ): ``pairs_per_face``
  adds that many pairs to a diagonal block per face neighbour (Section 4.3: one
  pair from the source term plus two per face flux, nine in the interior of a 2D
  grid, fewer on its boundary); ``random_pair_max > 0`` instead draws every
  block's count uniformly from ``0..random_pair_max`` with a generator of its
  own (seed + 7919), so the value draws keep their order.  ``r_diag`` and
  ``r_off`` of the returned workload are then the largest counts of each kind.

Value distributions: diagonal entries of diagonal blocks ``1/dt + |z|``; every
other S entry ``0.1 z``; ``u, v = z / sqrt(b)``; right-hand side ``z``; loss
weights ``W ~ U[0.5, 1.5]``; z standard normal.  Draw order: diagonal-block S,
off-diagonal S, U, V, right-hand side, W.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Workload:
    """Arrays of one synthetic block r1-sparse Jacobian plus a right-hand side."""

    Lx: int
    Ly: int
    N: int
    b: int
    r_diag: int
    r_off: int
    block_indptr: np.ndarray      # int32 [nc+1]
    block_indices: np.ndarray     # int32 [nnzb]
    d_indptr: np.ndarray          # int32 [b+1]
    d_indices: np.ndarray         # int32 [nnz_d]
    o_indptr: np.ndarray          # int32 [b+1]
    o_indices: np.ndarray         # int32 [nnz_o]
    pair_indptr: np.ndarray       # int32 [nnzb+1]
    S: np.ndarray                 # float64 [nnz_S]
    U: np.ndarray                 # float64 [n_pairs, b]
    V: np.ndarray                 # float64 [n_pairs, b]
    rhs: np.ndarray               # float64 [nc*b]
    W: np.ndarray                 # float64 [nc*b]
    seed: int = 0

    @property
    def n_cells(self) -> int:
        return self.Lx * self.Ly

    @property
    def nnzb(self) -> int:
        return int(self.block_indices.shape[0])

    @property
    def nnz_d(self) -> int:
        return int(self.d_indices.shape[0])

    @property
    def nnz_o(self) -> int:
        return int(self.o_indices.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(self.pair_indptr[-1])

    @property
    def n(self) -> int:
        return self.n_cells * self.b

    def is_diag_block(self) -> np.ndarray:
        """Boolean [nnzb]: True where block k sits on the diagonal."""
        rows = np.repeat(np.arange(self.n_cells, dtype=np.int64),
                         np.diff(self.block_indptr).astype(np.int64))
        return rows == self.block_indices

    def s_offsets(self) -> np.ndarray:
        """int64 [nnzb+1]: start of each block's S values in ``S``."""
        sizes = np.where(self.is_diag_block(), self.nnz_d, self.nnz_o).astype(np.int64)
        out = np.zeros(self.nnzb + 1, dtype=np.int64)
        np.cumsum(sizes, out=out[1:])
        return out


def mesh_adjacency(Lx: int, Ly: int):
    """Block CSR of a structured grid: self plus 4-neighbours, sorted ascending."""
    nc = Lx * Ly
    indptr = np.zeros(nc + 1, dtype=np.int32)
    cols = []
    for i in range(nc):
        iy, ix = divmod(i, Lx)
        row = []
        if iy > 0:
            row.append(i - Lx)
        if ix > 0:
            row.append(i - 1)
        row.append(i)
        if ix < Lx - 1:
            row.append(i + 1)
        if iy < Ly - 1:
            row.append(i + Lx)
        cols.extend(row)
        indptr[i + 1] = len(cols)
    return indptr, np.asarray(cols, dtype=np.int32)


def diag_pattern(N: int, w: int):
    """Diagonal-block pattern: level band +-w plus flow columns; dense flow rows."""
    b = N + 3
    indptr = [0]
    cols: list[int] = []
    for p in range(b):
        if p < N:
            row = list(range(max(0, p - w), min(N - 1, p + w) + 1)) + [N, N + 1, N + 2]
        else:
            row = list(range(b))
        cols.extend(row)
        indptr.append(len(cols))
    return np.asarray(indptr, dtype=np.int32), np.asarray(cols, dtype=np.int32)


def off_pattern(N: int):
    """Off-diagonal-block pattern: level diagonal plus flow columns; dense flow rows."""
    b = N + 3
    indptr = [0]
    cols: list[int] = []
    for p in range(b):
        row = [p, N, N + 1, N + 2] if p < N else list(range(b))
        cols.extend(row)
        indptr.append(len(cols))
    return np.asarray(indptr, dtype=np.int32), np.asarray(cols, dtype=np.int32)


def random_patterns(b: int, density: float, seed: int):
    """Two random b x b CSR patterns (diagonal-block one with every diagonal
    entry, neighbour one arbitrary but with every row non-empty), for exercising
    patterns outside the paper's family."""
    rng = np.random.default_rng(seed)
    out = []
    for with_diag in (True, False):
        indptr = [0]
        cols: list[int] = []
        for p in range(b):
            row = set(np.flatnonzero(rng.random(b) < density).tolist())
            if with_diag:
                row.add(p)
            if not row:
                row.add(int(rng.integers(b)))
            cols.extend(sorted(row))
            indptr.append(len(cols))
        out.append((np.asarray(indptr, dtype=np.int32), np.asarray(cols, dtype=np.int32)))
    return out


def pair_indptr_for(block_indptr, block_indices, r_diag: int, r_off: int) -> np.ndarray:
    """BR1-BSR ``pair_indptr``: r_diag pairs per diagonal block, r_off per other block."""
    block_indptr = np.asarray(block_indptr, dtype=np.int64)
    block_indices = np.asarray(block_indices, dtype=np.int64)
    nc = block_indptr.shape[0] - 1
    rows = np.repeat(np.arange(nc), np.diff(block_indptr))
    per_block = np.where(rows == block_indices, r_diag, r_off).astype(np.int64)
    out = np.zeros(block_indices.shape[0] + 1, dtype=np.int64)
    np.cumsum(per_block, out=out[1:])
    return out.astype(np.int32)


def _standard_normal(rng: np.random.Generator, n: int, chunk: int = 1 << 24) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    for s in range(0, n, chunk):
        rng.standard_normal(out=out[s:s + chunk])
    return out


def pair_counts_for(block_indptr, block_indices, r_diag: int, r_off: int,
                    pairs_per_face: int = 0, random_pair_max: int = 0, seed: int = 0) -> np.ndarray:
    """int64 [nnzb]: pairs of every block (see the module docstring)."""
    block_indptr = np.asarray(block_indptr, dtype=np.int64)
    block_indices = np.asarray(block_indices, dtype=np.int64)
    nc = block_indptr.shape[0] - 1
    deg = np.diff(block_indptr) - 1
    rows = np.repeat(np.arange(nc), np.diff(block_indptr))
    is_diag = rows == block_indices
    if random_pair_max > 0:
        rng = np.random.default_rng(seed + 7919)
        return rng.integers(0, random_pair_max + 1, size=block_indices.shape[0]).astype(np.int64)
    return np.where(is_diag, r_diag + pairs_per_face * deg[rows], r_off).astype(np.int64)


def make_workload(Lx: int, Ly: int | None = None, N: int = 10, w: int = 2,
                  r_diag: int = 2, r_off: int = 1, seed: int = 0, dt: float = 1e-3,
                  same_pattern: bool = False, random_density: float = 0.0,
                  pairs_per_face: int = 0, random_pair_max: int = 0) -> Workload:
    """Draw one workload; see the module docstring for shapes and distributions.
    ``random_density > 0`` replaces both patterns by random ones of that density."""
    Ly = Lx if Ly is None else Ly
    b = N + 3
    block_indptr, block_indices = mesh_adjacency(Lx, Ly)
    d_indptr, d_indices = diag_pattern(N, w)
    if same_pattern:
        o_indptr, o_indices = d_indptr.copy(), d_indices.copy()
    else:
        o_indptr, o_indices = off_pattern(N)
    if random_density > 0:
        (d_indptr, d_indices), (o_indptr, o_indices) = random_patterns(b, random_density, seed + 1000)
    nc = Lx * Ly
    nnzb = block_indices.shape[0]
    rows = np.repeat(np.arange(nc), np.diff(block_indptr))
    is_diag = rows == block_indices
    n_off = int(nnzb - nc)

    if pairs_per_face or random_pair_max:
        counts = pair_counts_for(block_indptr, block_indices, r_diag, r_off,
                                 pairs_per_face, random_pair_max, seed)
        pair_indptr = np.zeros(nnzb + 1, dtype=np.int64)
        np.cumsum(counts, out=pair_indptr[1:])
        pair_indptr = pair_indptr.astype(np.int32)
        r_diag = int(counts[is_diag].max(initial=0))
        r_off = int(counts[~is_diag].max(initial=0))
    else:
        pair_indptr = pair_indptr_for(block_indptr, block_indices, r_diag, r_off)
    n_pairs = int(pair_indptr[-1])

    nnz_d, nnz_o = d_indices.shape[0], o_indices.shape[0]
    rng = np.random.default_rng(seed)
    # 1. diagonal-block S, block order x pattern order
    zd = _standard_normal(rng, nc * nnz_d).reshape(nc, nnz_d)
    d_rows = np.repeat(np.arange(b), np.diff(d_indptr))
    on_diag = d_rows == d_indices
    sd = 0.1 * zd
    sd[:, on_diag] = 1.0 / dt + np.abs(zd[:, on_diag])
    # 2. off-diagonal S
    so = 0.1 * _standard_normal(rng, n_off * nnz_o).reshape(n_off, nnz_o)
    # 3. U, 4. V
    scale = 1.0 / math.sqrt(b)
    U = (_standard_normal(rng, n_pairs * b) * scale).reshape(n_pairs, b)
    V = (_standard_normal(rng, n_pairs * b) * scale).reshape(n_pairs, b)
    # 5. right-hand side, 6. loss weights
    rhs = _standard_normal(rng, nc * b)
    W = rng.uniform(0.5, 1.5, size=nc * b)

    # interleave the two S streams into block order, one block row at a time
    S = np.empty(nc * nnz_d + n_off * nnz_o, dtype=np.float64)
    pos = 0
    o = 0
    cols = block_indices
    for i in range(nc):
        for k in range(int(block_indptr[i]), int(block_indptr[i + 1])):
            if cols[k] == i:
                S[pos:pos + nnz_d] = sd[i]
                pos += nnz_d
            else:
                S[pos:pos + nnz_o] = so[o]
                pos += nnz_o
                o += 1
    assert pos == S.shape[0] and o == n_off

    return Workload(Lx=Lx, Ly=Ly, N=N, b=b, r_diag=r_diag, r_off=r_off,
                    block_indptr=block_indptr, block_indices=block_indices,
                    d_indptr=d_indptr, d_indices=d_indices,
                    o_indptr=o_indptr, o_indices=o_indices,
                    pair_indptr=pair_indptr, S=S, U=U, V=V,
                    rhs=rhs, W=W, seed=seed)


@dataclasses.dataclass
class FlowCase:
    """Inputs of the toy flow model whose HLL-flux Jacobian is built in r1-sparse form:
    per-species constants, source constants, pseudo time step, and two state fields
    (current iterate Q and previous time level Qn, [nc][b] with b = N + 3, variables
    rho_0..rho_{N-1}, u, v, T).  Nondimensional synthetic values (no rate data)."""

    Lx: int
    Ly: int
    N: int
    w: int
    r: np.ndarray           # [N] species gas constants R / M_k
    cv: np.ndarray          # [N] constant-volume specific heats
    e0: np.ndarray          # [N] level energies, e_k(T) = e0_k + cv_k T
    beta: np.ndarray        # [N] source weights of the reaction progress
    ws: np.ndarray          # [N] source stoichiometry
    K: np.ndarray           # [N][2w+1] level relaxation band, K[k][l - k + w]
    A: float
    theta: float
    dt: float
    Q: np.ndarray
    Qn: np.ndarray

    @property
    def b(self) -> int:
        return self.N + 3

    @property
    def n_cells(self) -> int:
        return self.Lx * self.Ly


def make_flow_case(Lx: int, Ly: int | None = None, N: int = 10, w: int = 2, seed: int = 0,
                   dt: float = 0.1, mach: float = 0.4) -> FlowCase:
    """Seeded constants and smooth state fields with 5% noise.  ``mach`` scales the
    velocity against a sound speed near 0.7: below 1 the HLL wave-speed bounds come
    from both sides of a face, above 1 they are clipped at zero on most faces."""
    Ly = Lx if Ly is None else Ly
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.25, 0.45, N)
    cv = rng.uniform(0.6, 1.2, N)
    e0 = 0.05 * np.arange(N) + rng.uniform(0.0, 0.02, N)
    beta = rng.uniform(0.0, 1.0, N)
    ws = 0.1 * rng.standard_normal(N)
    K = rng.uniform(0.0, 0.5, (N, 2 * w + 1))
    ix, iy = np.meshgrid(np.arange(Lx), np.arange(Ly))
    xs, ys = (ix.ravel() + 0.5) / Lx, (iy.ravel() + 0.5) / Ly
    nc = Lx * Ly
    Q = np.empty((nc, N + 3))
    T = 1.0 + 0.2 * np.cos(2 * np.pi * xs) * np.sin(np.pi * ys)
    rho = 1.0 + 0.3 * np.sin(np.pi * xs) * np.cos(np.pi * ys)
    pop = np.exp(-np.outer(1.0 / (0.5 + 0.3 * xs), e0 / 0.05 * 0.1))
    pop /= pop.sum(axis=1, keepdims=True)
    Q[:, :N] = rho[:, None] * pop * (1.0 + 0.05 * rng.standard_normal((nc, N)))
    Q[:, N] = mach * 0.7 * (1.0 + 0.3 * np.sin(2 * np.pi * ys)) * (1.0 + 0.05 * rng.standard_normal(nc))
    Q[:, N + 1] = mach * 0.7 * 0.4 * np.cos(np.pi * xs) * (1.0 + 0.05 * rng.standard_normal(nc))
    Q[:, N + 2] = T * (1.0 + 0.05 * rng.standard_normal(nc))
    Qn = Q * (1.0 + 0.01 * rng.standard_normal(Q.shape))
    return FlowCase(Lx=Lx, Ly=Ly, N=N, w=w, r=r, cv=cv, e0=e0, beta=beta, ws=ws, K=K,
                    A=1.0, theta=2.0, dt=dt, Q=Q, Qn=Qn)


# Workloads of the five measured configurations, named by what they are.
WORKLOADS = {
    # 16x16 cells, N=10 (b=13), band +-2, 2 diagonal / 1 neighbour pairs, seed 0
    "grid16_N10": dict(Lx=16, N=10, w=2, r_diag=2, r_off=1, seed=0),
    # 128x128 cells, N=60 (b=63), band +-2, 2 / 1 pairs, seed 1
    "grid128_N60": dict(Lx=128, N=60, w=2, r_diag=2, r_off=1, seed=1),
    # 256x256 cells, N=200 (b=203), band +-4, 3 / 1 pairs, seed 2
    "grid256_N200": dict(Lx=256, N=200, w=4, r_diag=3, r_off=1, seed=2),
    # 512x512 cells, N=60, FP32 operators inside FP64 flexible GMRES, seed 3
    "grid512_N60": dict(Lx=512, N=60, w=2, r_diag=2, r_off=1, seed=3),
    # 128x128 cells, N=60, adjoint gradients, seed 4
    "grid128_N60_adjoint": dict(Lx=128, N=60, w=2, r_diag=2, r_off=1, seed=4),
    # 128x128 cells, N=60, the paper's physical pair counts: 1 + 2 per face on
    # diagonal blocks (9 inside, 7 on edges, 5 in corners), 2 per neighbour block
    "grid128_N60_pairs9": dict(Lx=128, N=60, w=2, r_diag=1, r_off=2, pairs_per_face=2, seed=5),
}


def named_workload(name: str, **overrides) -> Workload:
    kw = dict(WORKLOADS[name])
    kw.update(overrides)
    return make_workload(**kw)
